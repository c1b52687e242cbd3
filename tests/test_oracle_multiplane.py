"""Pins of the oracle's multi-plane ray tracing (Sec. 1: several lens planes,
the mapping repeated plane by plane; a thick lens as a collection of thin
planes): reductions to the single-plane Eq. 1, superposition when no plane
sees another's deflection, the closed-form Einstein ring of two coaxial
masses on two planes, and the index structure of the distance ratios."""
import math

import numpy as np
import pytest

import oracle
from paper_2211_00354_gb300 import synth


def field(seed, n, ks=0.0, g=0.0, radius=6.0):
    rng = np.random.default_rng(seed)
    return (synth.uniform_disk(rng, n, radius), rng.uniform(0.5, 1.5, n), ks, g)


EMPTY = (np.zeros((0, 2)), np.zeros(0), 0.0, 0.0)


def test_one_plane_is_eq1():
    st, ms, ks, g = field(1, 300, 0.2, 0.1)
    x = synth.random_rays(2, 500, (-5, -5), (5, 5))
    y = oracle.multiplane_deflect([(st, ms, ks, g)], np.zeros((1, 1)), x)
    np.testing.assert_allclose(y, oracle.deflect(st, ms, ks, g, x), rtol=0, atol=1e-13)


@pytest.mark.parametrize("where", [0, 1])
def test_an_empty_plane_changes_nothing(where):
    p = field(3, 200, 0.1, -0.05)
    x = synth.random_rays(4, 400, (-4, -4), (4, 4))
    planes = [p, EMPTY] if where == 1 else [EMPTY, p]
    beta = np.array([[0.0, 0.37], [0.0, 0.0]])
    y, xp = oracle.multiplane_deflect(planes, beta, x, planes_out=True)
    # (a x - alpha against x - (alpha + (kappa + gamma) x): rounding order only)
    np.testing.assert_allclose(y, oracle.deflect(p[0], p[1], p[2], p[3], x), rtol=0, atol=1e-13)
    np.testing.assert_array_equal(xp[0], x)


def test_no_coupling_is_superposition():
    # beta = 0: no plane sees another's deflection, so the planes act as one
    # plane holding all their stars and the sum of their smooth fields
    a, b, c = field(5, 150, 0.1, 0.2), field(6, 120, 0.05, -0.1), field(7, 90, 0.0, 0.03)
    x = synth.random_rays(8, 300, (-5, -5), (5, 5))
    y = oracle.multiplane_deflect([a, b, c], np.zeros((3, 3)), x)
    st = np.concatenate([a[0], b[0], c[0]])
    ms = np.concatenate([a[1], b[1], c[1]])
    ref = oracle.deflect(st, ms, a[2] + b[2] + c[2], a[3] + b[3] + c[3], x)
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("m1,m2,beta", [(1.0, 0.5, 0.4), (0.3, 2.0, 0.8), (1.0, 1.0, 0.0)])
def test_einstein_ring_of_two_coaxial_masses(m1, m2, beta):
    # masses at the origin of planes 1 and 2; a ray at radius r reaches plane 2
    # at r (1 - beta m1 / r^2) and the source plane at
    # r - m1/r - m2 / (r (1 - beta m1 / r^2)); it lands on the axis when
    # u = r^2 solves u^2 - (m1 (1 + beta) + m2) u + beta m1^2 = 0
    B = m1 * (1 + beta) + m2
    u = 0.5 * (B + math.sqrt(B * B - 4 * beta * m1 * m1))
    r = math.sqrt(u)
    t = np.linspace(0, 2 * np.pi, 17)
    x = np.column_stack([r * np.cos(t), r * np.sin(t)])
    planes = [(np.zeros((1, 2)), np.array([m1]), 0.0, 0.0),
              (np.zeros((1, 2)), np.array([m2]), 0.0, 0.0)]
    y, xp = oracle.multiplane_deflect(planes, np.array([[0.0, beta], [0.0, 0.0]]), x,
                                      planes_out=True)
    assert np.abs(y).max() < 1e-13
    np.testing.assert_allclose(np.hypot(*xp[1].T), r * (1 - beta * m1 / u), rtol=1e-14)


def test_a_massless_middle_plane_leaves_the_outer_pair():
    # three planes with the middle one empty are two planes whose ratio is
    # beta[0, 2]; beta[0, 1] and beta[1, 2] must not enter
    a, c = field(9, 100, 0.05, 0.1), field(10, 80, 0.1, -0.05)
    x = synth.random_rays(11, 300, (-4, -4), (4, 4))
    b3 = np.array([[0.0, 0.9, 0.35], [0.0, 0.0, 0.6], [0.0, 0.0, 0.0]])
    y3 = oracle.multiplane_deflect([a, EMPTY, c], b3, x)
    y2 = oracle.multiplane_deflect([a, c], np.array([[0.0, 0.35], [0.0, 0.0]]), x)
    np.testing.assert_array_equal(y3, y2)


def test_two_planes_against_the_recursion_written_out():
    # plane 2 is evaluated where plane 1 sent the ray, not at the entry point
    a, b = field(12, 60, 0.1, 0.2), field(13, 70, 0.0, 0.1)
    x = synth.random_rays(14, 200, (-4, -4), (4, 4))
    beta = 0.55
    y = oracle.multiplane_deflect([a, b], np.array([[0.0, beta], [0.0, 0.0]]), x)
    y_at_entry = oracle.multiplane_deflect([a, b], np.zeros((2, 2)), x)
    assert np.abs(y - y_at_entry).max() > 1e-3
    # alpha_1 from the single-plane oracle, then plane 2 at x_2
    _, al1 = oracle.deflect(a[0], a[1], 0.0, 0.0, x, alpha=True)
    al1 = al1 + np.array([a[2] + a[3], a[2] - a[3]]) * x
    x2 = x - beta * al1
    _, al2 = oracle.deflect(b[0], b[1], 0.0, 0.0, x2, alpha=True)
    al2 = al2 + np.array([b[2] + b[3], b[2] - b[3]]) * x2
    np.testing.assert_allclose(y, x - al1 - al2, rtol=0, atol=1e-12)
