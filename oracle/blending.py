"""Blending, pseudo-deblending and gather sorting, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Ch. 2, Eqs ch2_blending and pseudodeblending_equ:
  * blending       b = Gamma D: every shot record D[i] ([receivers][nt]) is
                   added into one continuous record b ([receivers][nb]) from
                   its firing sample tau_i on,
                   b[r, t'] = sum_i D[i, r, t' - tau_i]  (0 <= t' - tau_i < nt);
  * pseudo-deblending D~ = Gamma^T b: each shot's window is cut back out,
                   D~[i, r, t] = b[r, tau_i + t]  (0 <= tau_i + t < nb, else 0),
                   which is the transpose of the blending;
  * sorting        common-shot gathers [shot][receiver][t] to common-receiver
                   gathers [receiver][shot][t] (ch. 2: the interference is
                   incoherent in the receiver domain) and back.
Readings where the thesis is silent: firing times are whole samples (the
dithered delays of the acquisition rounded to the sampling); samples of a
shot that fall outside the continuous record are dropped.
"""
import numpy as np


def blend(D, fire, nb):
    """b [nr][nb] from D [ns][nr][nt] and firing samples fire [ns]."""
    D = np.asarray(D, dtype=np.float64)
    ns, nr, nt = D.shape
    b = np.zeros((nr, nb))
    for i in range(ns):
        for t in range(nt):
            tp = int(fire[i]) + t
            if 0 <= tp < nb:
                b[:, tp] += D[i, :, t]
    return b


def pseudo_deblend(b, fire, nt):
    """D~ [ns][nr][nt] from b [nr][nb]: the transpose of ``blend``."""
    b = np.asarray(b, dtype=np.float64)
    nr, nb = b.shape
    ns = len(fire)
    D = np.zeros((ns, nr, nt))
    for i in range(ns):
        for t in range(nt):
            tp = int(fire[i]) + t
            if 0 <= tp < nb:
                D[i, :, t] = b[:, tp]
    return D


def sort_gathers(X):
    """[n0][n1][nt] -> [n1][n0][nt] (shot gathers <-> receiver gathers)."""
    X = np.asarray(X)
    out = np.empty((X.shape[1], X.shape[0], X.shape[2]), dtype=X.dtype)
    for i in range(X.shape[0]):
        for j in range(X.shape[1]):
            out[j, i] = X[i, j]
    return out
