"""Images of a point source and the lensed image of a Gaussian source on a
deflected ray grid (Sec. 2.5: the images of a background Gaussian source
behind a simulated halo, found from the deflections of a regular ray grid)
-- TEST INFRASTRUCTURE ONLY, plain float64 numpy.

``find_images`` follows the polygon model of the IPM (Sec. 2.3): the cell
(i, j) maps to the quadrilateral of its deflected corners (i, j), (i+1, j),
(i+1, j+1), (i, j+1).  A cell holds an image of the point source beta when
beta lies in the bounding box of those corners and the closed polygon winds
around it (crossing rule, each orientation product an IEEE-rounded float64
expression).  Inside such a cell the corners' bilinear interpolation is
inverted by Newton's method (a fixed 20 steps from the cell centre, cell
coordinates kept within [-1, 2]); the image sits at that point and its
signed magnification is h^2 over the determinant of the bilinear map's
Jacobian there (Sec. 2.3: magnification as the ratio of areas).  A cell
that holds a point mass maps to a polygon around its whole neighbourhood
and reports the mass's infinitely demagnified image (|mu| ~ 1e-11 for a
unit mass in a cell of 0.004).

``source_image`` is the surface brightness exp(-|y - beta|^2 / 2 sigma^2) of
a Gaussian source seen at each ray (lensing conserves surface brightness).
"""
from __future__ import annotations

import numpy as np

NEWTON_STEPS = 20


def winding_numbers(y, beta):
    """Winding number of each cell's deflected quadrilateral around beta
    (0 outside the corners' bounding box).  y: (ny+1, nx+1, 2)."""
    y = np.asarray(y, dtype=np.float64)
    b1, b2 = float(beta[0]), float(beta[1])
    q = [y[:-1, :-1], y[:-1, 1:], y[1:, 1:], y[1:, :-1]]
    w = np.zeros(q[0].shape[:2], dtype=np.int64)
    for e in range(4):
        a, b = q[e], q[(e + 1) % 4]
        ax, ay, bx, by = a[..., 0], a[..., 1], b[..., 0], b[..., 1]
        # (b - a) x (beta - a), each product and difference rounded once
        cr = (bx - ax) * (b2 - ay) - (b1 - ax) * (by - ay)
        up = (ay <= b2) & (b2 < by) & (cr > 0)
        down = (by <= b2) & (b2 < ay) & (cr < 0)
        w += up.astype(np.int64) - down.astype(np.int64)
    xs = np.stack([c[..., 0] for c in q])
    ys = np.stack([c[..., 1] for c in q])
    inside = (xs.min(0) <= b1) & (b1 <= xs.max(0)) & (ys.min(0) <= b2) & (b2 <= ys.max(0))
    return np.where(inside, w, 0)


def invert_bilinear(q0, q1, q2, q3, beta, steps=NEWTON_STEPS):
    """(s, t, det J): the cell coordinates where the bilinear interpolation
    p(s, t) = q0 + s e + t f + s t g (e = q1 - q0, f = q3 - q0,
    g = q0 - q1 + q2 - q3) meets beta, by Newton's method from (1/2, 1/2)."""
    q0, q1, q2, q3 = (np.asarray(v, dtype=np.float64) for v in (q0, q1, q2, q3))
    e, f, g = q1 - q0, q3 - q0, q0 - q1 + q2 - q3
    s = t = 0.5
    for _ in range(steps):
        js = e + t * g          # dp/ds
        jt = f + s * g          # dp/dt
        r = np.asarray(beta, dtype=np.float64) - (q0 + s * e + t * f + s * t * g)
        det = js[0] * jt[1] - jt[0] * js[1]
        if det == 0.0:
            break
        s = min(max(s + (r[0] * jt[1] - jt[0] * r[1]) / det, -1.0), 2.0)
        t = min(max(t + (js[0] * r[1] - r[0] * js[1]) / det, -1.0), 2.0)
    js = e + t * g
    jt = f + s * g
    return s, t, js[0] * jt[1] - jt[0] * js[1]


def find_images(y, x0, y0, h, beta):
    """Image cells of the point source beta: a list of (cell, x1, x2, mu)
    sorted by cell = j * nx + i."""
    y = np.asarray(y, dtype=np.float64)
    ny, nx = y.shape[0] - 1, y.shape[1] - 1
    w = winding_numbers(y, beta)
    out = []
    for j, i in zip(*np.nonzero(w)):
        s, t, det = invert_bilinear(y[j, i], y[j, i + 1], y[j + 1, i + 1], y[j + 1, i], beta)
        mu = h * h / det if det != 0.0 else np.inf
        out.append((int(j) * nx + int(i), x0 + (i + s) * h, y0 + (j + t) * h, mu))
    return out


def source_image(y, beta, sigma):
    """exp(-|y_r - beta|^2 / (2 sigma^2)) at every ray."""
    y = np.asarray(y, dtype=np.float64).reshape(-1, 2)
    d2 = (y[:, 0] - beta[0]) ** 2 + (y[:, 1] - beta[1]) ** 2
    return np.exp(-d2 / (2.0 * sigma * sigma))
