"""Finite-difference stencils used as stencil workloads (taps only, no arithmetic).

"Order r" is the second-derivative central difference of radius r (accuracy
2r) applied along both axes, i.e. the 2-D Laplacian on a cross of 4r + 1
points.  Coefficients are the standard central-difference weights
(B. Fornberg, "Generation of finite difference formulas on arbitrarily spaced
grids", Math. Comp. 51, 1988).
"""
from fractions import Fraction as F

# weights of f(x + i h), i = -r..r, for f'' at accuracy 2r
SECOND_DERIVATIVE = {
    1: [F(1), F(-2), F(1)],
    2: [F(-1, 12), F(4, 3), F(-5, 2), F(4, 3), F(-1, 12)],
    3: [F(1, 90), F(-3, 20), F(3, 2), F(-49, 18), F(3, 2), F(-3, 20), F(1, 90)],
    4: [F(-1, 560), F(8, 315), F(-1, 5), F(8, 5), F(-205, 72), F(8, 5), F(-1, 5), F(8, 315), F(-1, 560)],
}


def fd_laplacian(order: int):
    """Taps (dy, dx, w) of the order-r 2-D Laplacian (centre weight summed)."""
    c = SECOND_DERIVATIVE[order]
    r = order
    taps = {}
    for i, w in enumerate(c):
        d = i - r
        taps[(d, 0)] = taps.get((d, 0), F(0)) + w
        taps[(0, d)] = taps.get((0, d), F(0)) + w
    return [(dy, dx, float(w)) for (dy, dx), w in sorted(taps.items())]
