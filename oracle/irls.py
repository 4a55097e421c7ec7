"""Robust l_p - l_q Radon inversion by IRLS with an inner CGLS, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows ch. 4, "Robust Radon transform":
  * cost J = ||d - L m||_p^p + mu ||m||_q^q                  (Eq. ch4_cost_fn)
  * diagonal weights [W_x]_ii = 1 / sqrt(|x_i|^(2-p)), floored at eps
    (the W_m and W_r definitions that follow it), read with |x_i|
  * eps_r = b_r MAD(r) / 0.6745, b_r = 1.345, MAD = Med(|r - Med(r)|)
                                                             (Eq. ch4_epcilon_r)
  * eps_m = b_m max|m| / 100
  * weighted cost J = ||W_r r||^2 + mu ||W_m m||^2            (Eq. equ:10)
    in standard form with u = W_m m:
    J = ||W_r (L W_m^-1 u - d)||^2 + mu ||u||^2               (Eq. equ:11)
  * inner conjugate gradients (CGLS on the normal equations), outer weight
    update, stop on relative misfit change < tol or at the iteration cap;
    mu = 0 by default, the CG count acting as the regulariser.
Quality: Q = 10 log10(||d_o||^2 / ||d_o - d_r||^2)   (Eqs ch4_Qpd, ch4_Qr).

Readings where the thesis is silent: W = I at the first outer iteration; CGLS is
warm-started from u0 = W_m m_prev; median of an even count is the mean of the
two middle order statistics; MAD = 0 falls back to eps_r = 1e-6 max|r| (then
1e-30); max|m| = 0 gives W_m = I; the misfit is J_k = sum |r_i|^p over the
live samples after outer iteration k.
"""
import numpy as np


def median(x):
    x = np.sort(np.asarray(x, dtype=np.float64).ravel())
    n = x.size
    if n == 0:
        return 0.0
    if n % 2:
        return float(x[n // 2])
    return 0.5 * (float(x[n // 2 - 1]) + float(x[n // 2]))


def mad(x):
    """MAD(r) = Med(|r - Med(r)|)  (ch. 4, after Eq. ch4_epcilon_r)."""
    x = np.asarray(x, dtype=np.float64).ravel()
    return median(np.abs(x - median(x)))


def eps_residual(r_live, b_r=1.345):
    """eps_r = b_r MAD / 0.6745 (Eq. ch4_epcilon_r) with the zero-MAD guard."""
    e = b_r * mad(r_live) / 0.6745
    if e == 0.0:
        e = 1e-6 * float(np.max(np.abs(r_live))) if np.size(r_live) else 0.0
    if e == 0.0:
        e = 1e-30
    return e


def eps_model(m, b_m=1.0):
    """eps_m = b_m max|m| / 100; 0 when m == 0 (W_m = I is used then)."""
    return b_m * float(np.max(np.abs(m))) / 100.0


def weight(x, eps, p):
    """[W]_ii = 1/sqrt(max(|x_i|, eps)^(2-p)) = max(|x_i|, eps)^((p-2)/2)."""
    return np.maximum(np.abs(x), eps) ** ((p - 2.0) / 2.0)


def weight_inverse(x, eps, q):
    """[W]^-1_ii = max(|x_i|, eps)^((2-q)/2): the inverse model weight W_m^-1."""
    return np.maximum(np.abs(x), eps) ** ((2.0 - q) / 2.0)


def cgls(A, AT, b, x0, niter, mu=0.0):
    """Conjugate gradients on min ||A x - b||^2 + mu ||x||^2 (normal equations).

    Returns (x, n_forward_applies, n_adjoint_applies).
    """
    x = np.array(x0, dtype=np.float64, copy=True)
    nf = na = 0
    if np.any(x):
        r = b - A(x)
        nf += 1
    else:
        r = np.array(b, dtype=np.float64, copy=True)
    s = AT(r) - mu * x
    na += 1
    p = s.copy()
    gamma = float(np.vdot(s, s))
    for _ in range(niter):
        q = A(p)
        nf += 1
        delta = float(np.vdot(q, q)) + mu * float(np.vdot(p, p))
        if delta <= 0.0 or gamma <= 0.0:
            break
        alpha = gamma / delta
        x += alpha * p
        r -= alpha * q
        s = AT(r) - mu * x
        na += 1
        gamma_new = float(np.vdot(s, s))
        beta = gamma_new / gamma
        gamma = gamma_new
        p = s + beta * p
    return x, nf, na


def irls(fwd, adj, d, n_outer, n_cg, p=1.0, q=1.0, b_r=1.345, b_m=1.0, mu=0.0,
         live=None, eps_r_fixed=None, eps_m_fixed=None, tol=0.0, warm_start=True,
         m0=None, wr0=None):
    """IRLS for min ||d - L m||_p^p + mu ||m||_q^q (ch. 4).

    fwd(m) -> data and adj(d) -> model are the (masked) operator pair; ``live``
    is a boolean array over data samples used for MAD and misfit (all True if
    None).  Returns (m, report) with report = dict(misfit=[...], outer_done,
    applies_fwd, applies_adj, d_model = fwd(m)).

    Warm start (an extension for learned initial guesses; the thesis always
    starts cold): with m0 the first outer iteration already reweights, W_m from
    m0 and W_r from the residual of m0 (or wr0 when given); with only wr0 the
    first iteration uses W_r = wr0 and W_m = I.
    """
    d = np.asarray(d, dtype=np.float64)
    live = np.ones(d.shape, dtype=bool) if live is None else np.asarray(live, dtype=bool)
    m = np.zeros_like(adj(np.zeros_like(d)))
    nf, na = 0, 0
    misfit = []
    Wr = np.ones_like(d)
    Wm_inv = np.ones_like(m)
    y = None
    if m0 is not None:
        m = np.array(m0, dtype=np.float64).reshape(m.shape)
        y = fwd(m)
        nf += 1
    for k in range(n_outer):
        if k > 0 or m0 is not None:
            if k == 0 and wr0 is not None:
                Wr = np.asarray(wr0, dtype=np.float64)
            else:
                r = np.where(live, d - y, 0.0)
                er = eps_r_fixed if eps_r_fixed is not None else eps_residual(r[live], b_r)
                Wr = weight(r, er, p)
            em = eps_m_fixed if eps_m_fixed is not None else eps_model(m, b_m)
            Wm_inv = weight_inverse(m, em, q) if em > 0.0 else np.ones_like(m)
        elif wr0 is not None:
            Wr = np.asarray(wr0, dtype=np.float64)

        def A(u, Wr=Wr, Wm_inv=Wm_inv):
            return Wr * fwd(Wm_inv * u)

        def AT(r, Wr=Wr, Wm_inv=Wm_inv):
            return Wm_inv * adj(Wr * r)

        u0 = m / Wm_inv if warm_start else np.zeros_like(m)
        u, f1, a1 = cgls(A, AT, Wr * np.where(live, d, 0.0), u0, n_cg, mu)
        nf += f1
        na += a1
        m = Wm_inv * u
        y = fwd(m)
        nf += 1
        rr = np.where(live, d - y, 0.0)
        misfit.append(float(np.sum(np.abs(rr[live]) ** p)))
        if tol > 0.0 and k > 0 and misfit[-2] > 0.0 and \
                abs(misfit[-1] - misfit[-2]) / misfit[-2] < tol:
            break
    return m, dict(misfit=misfit, outer_done=len(misfit), applies_fwd=nf,
                   applies_adj=na, d_model=y)


def q_db(d_orig, d_test):
    """Q = 10 log10(||d_orig||^2 / ||d_orig - d_test||^2)   (Eqs ch4_Qpd, ch4_Qr)."""
    d_orig = np.asarray(d_orig, dtype=np.float64)
    e = d_orig - np.asarray(d_test, dtype=np.float64)
    return 10.0 * np.log10(np.sum(d_orig * d_orig) / np.sum(e * e))
