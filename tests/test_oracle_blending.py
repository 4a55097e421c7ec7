"""Pins for the blending / pseudo-deblending / sorting oracle (ch. 2, Eqs
ch2_blending and pseudodeblending_equ): the transpose identity, the closed
form of shots that do not overlap (the record is their concatenation and
pseudo-deblending restores them exactly), hand values of an overlap, and the
sort being an involution that moves element (i, j, t) to (j, i, t)."""
import numpy as np

from oracle import blending


def test_pseudo_deblending_is_the_transpose_of_blending():
    rng = np.random.default_rng(0)
    D = rng.standard_normal((7, 3, 20))
    fire = np.array([-5, 0, 8, 15, 15, 30, 41])          # overlaps, a negative start, a cut tail
    nb = 50
    b = rng.standard_normal((3, nb))
    lhs = np.vdot(blending.blend(D, fire, nb), b)
    rhs = np.vdot(D, blending.pseudo_deblend(b, fire, 20))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_shots_without_overlap_concatenate_and_come_back():
    rng = np.random.default_rng(1)
    D = rng.standard_normal((4, 2, 10))
    fire = np.array([0, 10, 20, 30])
    b = blending.blend(D, fire, 40)
    assert np.array_equal(b, np.concatenate(list(D), axis=1))
    assert np.array_equal(blending.pseudo_deblend(b, fire, 10), D)


def test_overlap_hand_values():
    D = np.zeros((2, 1, 4))
    D[0, 0] = [1.0, 2.0, 3.0, 4.0]
    D[1, 0] = [10.0, 20.0, 30.0, 40.0]
    b = blending.blend(D, [0, 2], 7)
    assert np.array_equal(b[0], [1.0, 2.0, 13.0, 24.0, 30.0, 40.0, 0.0])
    Dt = blending.pseudo_deblend(b, [0, 2], 4)
    assert np.array_equal(Dt[0, 0], [1.0, 2.0, 13.0, 24.0])       # shot 0 with shot 1's head
    assert np.array_equal(Dt[1, 0], [13.0, 24.0, 30.0, 40.0])     # shot 1 with shot 0's tail


def test_sort_moves_elements_and_is_an_involution():
    X = np.arange(3 * 5 * 4).reshape(3, 5, 4)
    Y = blending.sort_gathers(X)
    assert Y.shape == (5, 3, 4)
    assert Y[4, 2, 3] == X[2, 4, 3] and Y[0, 1, 2] == X[1, 0, 2]
    assert np.array_equal(blending.sort_gathers(Y), X)
