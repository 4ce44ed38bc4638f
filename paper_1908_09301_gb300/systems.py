"""Named three-component quadratic systems for ``Context.set_system``.

The paper's method applies to any right-hand side that automatic
differentiation handles (Sec. 2, after Fig. 1): sums and products give
Cauchy sums like those of Eq. (3).  A system is a dict:

* ``params``: parameter strings (decimal or ``a/b``), parameter p is the
  p-th one;
* ``fixed``: (target, neg, p, j) terms: p * x_j, the lone x_j (p = -1) or
  the constant p (j = -1);
* ``quad``: (target, neg, i, j) Cauchy products x_i * x_j.

Components 0, 1, 2 are x, y, z.
"""

# x' = sigma (y - x), y' = R x - y - x z, z' = x y - b z (Eq. (1))
LORENZ = {
    "params": ["10", "28", "8/3"],
    "fixed": [(0, 0, 0, 1), (0, 1, 0, 0), (1, 0, 1, 0), (1, 1, -1, 1), (2, 1, 2, 2)],
    "quad": [(1, 1, 0, 2), (2, 0, 0, 1)],
}

# Roessler: x' = -y - z, y' = x + a y, z' = b + z x - c z (a, b, c = 0.2, 0.2, 5.7)
ROESSLER = {
    "params": ["0.2", "0.2", "5.7"],
    "fixed": [(0, 1, -1, 1), (0, 1, -1, 2), (1, 0, -1, 0), (1, 0, 0, 1), (2, 0, 1, -1), (2, 1, 2, 2)],
    "quad": [(2, 0, 2, 0)],
}

# Chen: x' = a (y - x), y' = (c - a) x - x z + c y, z' = x y - b z (a, b, c = 35, 3, 28)
CHEN = {
    "params": ["35", "3", "28", "-7"],
    "fixed": [(0, 0, 0, 1), (0, 1, 0, 0), (1, 0, 3, 0), (1, 0, 2, 1), (2, 1, 1, 2)],
    "quad": [(1, 1, 0, 2), (2, 0, 0, 1)],
}

SYSTEMS = {"lorenz": LORENZ, "roessler": ROESSLER, "chen": CHEN}
