"""Algorithm 1 of the paper: solver-free ADMM on the model of Eq. (OurModel).

Notation follows the paper: ``x`` is the global vector, ``z`` the local
copies stacked as z = [x_1; ...; x_S], ``lam`` the stacked duals and ``B``
the stacked 0-1 consensus matrix of Section IV-C.

One iteration (Algorithm 1, global -> local -> dual):

* global update, Eq. (global_sparse):
      xhat = -(1/rho)(B^T B)^{-1} c + (B^T B)^{-1} B^T (z - lam/rho),
      x    = min(max(xhat, xlo), xhi);
  (Eq. closed_1 as printed omits the factor rho on the copy sum; the
  stacked form is the one that follows from minimizing Eq. ADMM-1.)
* local update, Eq. (closed_2): d_s = -rho B_s x - lam_s,
      x_s = (1/rho) Abar_s d_s + bbar_s;
* dual update, Eq. (ADMM-3 / dual_sparse): lam += rho (B x - z).

Termination, Eq. (termination): pres = sqrt(sum_s ||B_s x - x_s||^2),
dres = rho sqrt(sum_s ||B_s^T (x_s - x_s_prev)||^2),
eps_prim = eps_rel max(sqrt(sum_s ||B_s x||^2), sqrt(sum_s ||x_s||^2)),
eps_dual = eps_rel sqrt(sum_s ||B_s^T lam_s||^2).
Readings: the printed form keeps the sum over s outside the norm ("paper");
the "textbook" option puts it inside (rho ||B^T dz||, eps_rel ||B^T lam||).
At the first iteration the previous local vector is the initial one.
Criteria: ABS (pres <= eps_abs_prim and dres <= eps_abs_dual), REL (the
paper's relative test), BOTH, NEVER.

Initialization (Section V-A): lam = 0; each local entry is 1 if it copies a
squared voltage magnitude, the midpoint of its global variable's bounds if
both are finite, and 0 otherwise.

Residual balancing (option): Section III-D names residual balancing as an
acceleration that reduces the iteration count.  The rule used here is the
standard one for unscaled duals: at a residual check that does not stop,
rho <- tau * rho when pres > mu * dres, rho <- rho / tau when dres > mu * pres;
lambda is kept, and Abar_s, bbar_s do not depend on rho.  Checks happen every
``check_every`` iterations counted from the start of the run.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

from .model import VAR_W

CRIT_ABS, CRIT_REL, CRIT_BOTH, CRIT_NEVER = 0, 1, 2, 3
RES_PAPER, RES_TEXTBOOK = 0, 1


@dataclasses.dataclass
class Residuals:
    pres: float
    dres: float
    eps_prim: float
    eps_dual: float


class ADMM:
    def __init__(self, model, pre, rho: float):
        self.model = model
        self.rho = float(rho)
        self.gidx = np.concatenate([c.gvars for c in model.comps]).astype(np.int64)
        sizes = np.array([len(c.gvars) for c in model.comps], dtype=np.int64)
        self.comp_ptr = np.concatenate([[0], np.cumsum(sizes)])
        nl = len(self.gidx)
        self.B = sp.csr_matrix((np.ones(nl), (np.arange(nl), self.gidx)), shape=(nl, model.n))
        self.BT = self.B.T.tocsr()
        self.k = np.asarray(self.B.sum(axis=0)).ravel()          # diag(B^T B)
        if np.any(self.k < 1):
            raise ValueError("a global variable has no local copy")
        self.Abar = (sp.block_diag([sp.csr_matrix(a) for a in pre.Abar], format="csr")
                     if nl else sp.csr_matrix((0, 0)))
        self.bbar = np.concatenate(pre.bbar) if nl else np.zeros(0)
        self.c = model.c
        self.lo = model.lo
        self.hi = model.hi
        self.init()

    # Section V-A
    def initial_local(self) -> np.ndarray:
        lo, hi = self.lo[self.gidx], self.hi[self.gidx]
        z = np.zeros(len(self.gidx))
        both = np.isfinite(lo) & np.isfinite(hi)
        z[both] = 0.5 * (lo[both] + hi[both])
        z[self.model.vtype[self.gidx] == VAR_W] = 1.0
        return z

    def init(self):
        self.z = self.initial_local()
        self.lam = np.zeros(len(self.gidx))
        self.x = np.zeros(self.model.n)
        self.t = 0

    # Eq. (global_sparse)
    def global_update(self) -> np.ndarray:
        rho = self.rho
        xhat = -(1.0 / rho) * self.c / self.k + (self.BT @ (self.z - self.lam / rho)) / self.k
        return np.minimum(np.maximum(xhat, self.lo), self.hi)

    # Eq. (closed_2)
    def local_update(self, x: np.ndarray) -> np.ndarray:
        d = -self.rho * (self.B @ x) - self.lam
        return (self.Abar @ d) / self.rho + self.bbar

    def residuals(self, Bx, z, z_prev, lam, form=RES_PAPER, eps_rel=1e-3) -> Residuals:
        pres = float(np.sqrt(np.sum((Bx - z) ** 2)))
        if form == RES_PAPER:
            # ||B_s^T v|| = ||v|| since B_s has one 1 per row and at most one per column
            dres = self.rho * float(np.sqrt(np.sum((z - z_prev) ** 2)))
            dnorm = float(np.sqrt(np.sum(lam ** 2)))
        else:
            dres = self.rho * float(np.linalg.norm(self.BT @ (z - z_prev)))
            dnorm = float(np.linalg.norm(self.BT @ lam))
        eps_prim = eps_rel * max(float(np.linalg.norm(Bx)), float(np.linalg.norm(z)))
        return Residuals(pres, dres, eps_prim, eps_rel * dnorm)

    def step(self, form=RES_PAPER, eps_rel=1e-3) -> Residuals:
        """One iteration of Algorithm 1 (global, local, dual) and its residuals."""
        x = self.global_update()
        z_prev = self.z
        z = self.local_update(x)
        Bx = self.B @ x
        lam = self.lam + self.rho * (Bx - z)          # Eq. (ADMM-3)
        self.x, self.z, self.lam = x, z, lam
        self.t += 1
        return self.residuals(Bx, z, z_prev, lam, form, eps_rel)

    def run(self, max_iter: int, *, eps_abs_prim=1e-4, eps_abs_dual=1e-4, eps_rel=1e-3,
            criterion=CRIT_ABS, form=RES_PAPER, snapshots=(), history=False,
            check_every=1, adaptive_rho=False, rb_mu=10.0, rb_tau=2.0):
        """Iterate until the criterion holds (tested every ``check_every``
        iterations and at max_iter) or max_iter; returns a dict with the final
        residuals, iteration count, optional per-iteration residual history,
        (x, z, lam) copies at the iterations in ``snapshots`` and the final
        rho (residual balancing changes it at checks that do not stop)."""
        snaps = {}
        hist = []
        want = set(int(s) for s in snapshots)
        converged = False
        res = None
        first_rel = None
        changes = 0
        for k in range(1, max_iter + 1):
            res = self.step(form, eps_rel)
            if history:
                hist.append((res.pres, res.dres, res.eps_prim, res.eps_dual))
            if self.t in want:
                snaps[self.t] = (self.x.copy(), self.z.copy(), self.lam.copy())
            if k % check_every and k != max_iter:
                continue
            ok_abs = res.pres <= eps_abs_prim and res.dres <= eps_abs_dual
            ok_rel = res.pres <= res.eps_prim and res.dres <= res.eps_dual
            if ok_rel and first_rel is None:
                first_rel = self.t
            if ((criterion == CRIT_ABS and ok_abs) or (criterion == CRIT_REL and ok_rel)
                    or (criterion == CRIT_BOTH and ok_abs and ok_rel)):
                converged = True
                break
            if adaptive_rho and k != max_iter:
                if res.pres > rb_mu * res.dres:
                    self.rho *= rb_tau
                    changes += 1
                elif res.dres > rb_mu * res.pres:
                    self.rho /= rb_tau
                    changes += 1
        return dict(iters=self.t, converged=converged, res=res, snapshots=snaps,
                    history=np.array(hist), first_rel=first_rel, rho=self.rho, rho_changes=changes,
                    objective=float(self.c @ self.x))

    def objective(self) -> float:
        return float(self.c @ self.x)


def dual_certificate(model, pre, solver: ADMM):
    """LP dual value implied by the ADMM duals (a lower bound at a dual-feasible
    point) and the reduced costs.

    At a fixed point lam_s = A_s^T mu_s; with y_s = (A_s A_s^T)^{-1} A_s lam_s,
    r = c + sum_s B_s^T A_s^T y_s and g = -sum_s b_s^T y_s + sum_i min(lo_i r_i,
    hi_i r_i) (free variables must have r_i = 0; their |r_i| is returned)."""
    n = model.n
    r = model.c.astype(np.float64).copy()
    g = 0.0
    for s, comp in enumerate(model.comps):
        A, b = pre.Ared[s], pre.bred[s]
        if A.shape[0] == 0:
            continue
        lam_s = solver.lam[solver.comp_ptr[s]:solver.comp_ptr[s + 1]]
        y = np.linalg.solve(A @ A.T, A @ lam_s)
        np.add.at(r, comp.gvars, A.T @ y)
        g -= float(b @ y)
    free_res = 0.0
    for i in range(n):
        lo, hi = model.lo[i], model.hi[i]
        if np.isfinite(lo) and np.isfinite(hi):
            g += min(lo * r[i], hi * r[i])
        elif np.isfinite(lo):
            g += lo * r[i] if r[i] >= 0 else 0.0
            free_res = max(free_res, max(0.0, -r[i]))
        elif np.isfinite(hi):
            g += hi * r[i] if r[i] <= 0 else 0.0
            free_res = max(free_res, max(0.0, r[i]))
        else:
            free_res = max(free_res, abs(r[i]))
    return dict(dual=g, primal=float(model.c @ solver.x), reduced_cost=r, free_residual=free_res)


def solve_feeder(feeder, rho=100.0, max_iter=100000, **kw):
    """Build, precompute and run Algorithm 1 on one feeder (convenience)."""
    from .model import build_feeder
    from .precompute import precompute
    model = build_feeder(feeder)
    pre = precompute(model)
    solver = ADMM(model, pre, rho)
    out = solver.run(max_iter, **kw)
    return model, pre, solver, out
