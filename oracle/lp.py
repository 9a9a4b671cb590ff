"""The centralized LP of Eq. (LP_model), solved by HiGHS through scipy.

min c^T x  s.t.  A x = b (the stacked component rows A_s B_s),
                 xlo <= x <= xhi.
Used only to pin the ADMM fixed point (objective value) on small feeders.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import linprog

from .model import stacked_A


def solve_lp(model):
    A, b = stacked_A(model)
    bounds = [(None if not np.isfinite(l) else l, None if not np.isfinite(h) else h)
              for l, h in zip(model.lo, model.hi)]
    res = linprog(model.c, A_eq=A, b_eq=b, bounds=bounds, method="highs",
                  options=dict(primal_feasibility_tolerance=1e-10,
                               dual_feasibility_tolerance=1e-10))
    return res
