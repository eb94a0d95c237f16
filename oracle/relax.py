"""Local relaxation of one structure (Sec. II C): the level between the DE search and the
energy/force evaluation.

TEST INFRASTRUCTURE (oracle): only tests/ and bench.py's CPU legs use it; it imports
nothing from the product package.  Plain FP64 NumPy, written from Sec. II C:

* PCG: nonlinear preconditioned conjugate gradients whose preconditioner is an
  approximate inverse Hessian.  A classical force field is first fitted to reproduce the
  DFT atomic forces (here a Morse pair potential, parameters (D, a, r0), fitted by
  Levenberg-Marquardt to the force sets of the last HIST evaluated configurations); its Hessian is
  the second-order finite difference of the fitted energy (central differences of the
  fitted forces); the three zero eigenvalues of the translations are dropped and
  H^-1 = sum_j V_j V_j^T / tau_j over the others.  The fit and the preconditioner are
  renewed during the relaxation (every `refit` search directions).
* CG: the same nonlinear CG without the force field (preconditioner I / kappa0).
* BFGS: quasi-Newton on the inverse Hessian, started from I / kappa0.

The paper leaves the force field, the fit, the line minimisation and the step control
open; the readings taken here (written out in the functions below) are the ones the
GPU path's driver (csrc/relax.cpp) implements independently.

Pins (tests/test_oracle_relax.py): the fit recovers the parameters of forces that come
from a Morse potential; the truncated inverse annihilates the translations and inverts H
on the rest; a Morse dimer and an equilateral trimer relax to the analytic minimum
(r = r0); on a harmonic model (P = exact inverse) PCG lands on the minimum in one step.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Tuple

import numpy as np

KAPPA0 = 0.5        # Ha/bohr^2: stiffness behind the unpreconditioned trial steps (CG, BFGS)
FLOOR = 0.02        # kept eigenvalues of the force-field Hessian: |tau| >= FLOOR max|tau|
H_FD = 1e-3         # bohr: central-difference step of the force-field Hessian
HIST = 64           # the fit uses the last HIST evaluated configurations


# ---------------------------------------------------------------------------
# classical force field: shifted-force Morse pairs over periodic images
# ---------------------------------------------------------------------------
def morse_dphi(theta, r):
    """phi'(r) of phi(r) = D [exp(-2a(r - r0)) - 2 exp(-a(r - r0))]."""
    D, a, r0 = theta
    e = np.exp(-a * (r - r0))
    return 2.0 * D * a * (e - e * e)


def image_vectors(cell, rc):
    """Lattice translations L = n . A with |L| possibly < rc + the cell diagonal."""
    cell = np.asarray(cell, float)
    inv = np.linalg.inv(cell)
    # perpendicular widths: 1 / |row of inv^T|
    widths = 1.0 / np.linalg.norm(inv.T, axis=1)
    nmax = [int(np.ceil(rc / w)) + 1 for w in widths]
    ns = np.array([(i, j, k) for i in range(-nmax[0], nmax[0] + 1) for j in range(-nmax[1], nmax[1] + 1)
                   for k in range(-nmax[2], nmax[2] + 1)], float)
    return ns @ cell


def morse_dphi_grad(theta, r):
    """d phi'(r) / d(D, a, r0) (each an array over r)."""
    D, a, r0 = theta
    e = np.exp(-a * (r - r0))
    g = e - e * e
    h = 1.0 - 2.0 * e
    return 2.0 * a * g, 2.0 * D * g - 2.0 * D * a * h * (r - r0) * e, 2.0 * D * a * h * a * e


def ff_forces_jac(theta, cell, pos, rc):
    """The force field's forces and their derivatives dF_i/dtheta_k (natoms x 3 x 3),
    differentiating each pair term (phi'(r) - phi'(rc)) rv / r analytically."""
    pos = np.asarray(pos, float)
    n = len(pos)
    Ls = image_vectors(cell, rc)
    dc = morse_dphi(theta, rc)
    gc = morse_dphi_grad(theta, np.array(rc))
    F = np.zeros((n, 3))
    J = np.zeros((n, 3, 3))
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            rv = pos[j][None, :] + Ls - pos[i][None, :]
            r = np.linalg.norm(rv, axis=1)
            m = (r < rc) & (r > 1e-12)
            rr = r[m]
            u = rv[m] / rr[:, None]
            F[i] += ((morse_dphi(theta, rr) - dc)[:, None] * u).sum(axis=0)
            g = morse_dphi_grad(theta, rr)
            for k in range(3):
                J[i, :, k] += ((g[k] - gc[k])[:, None] * u).sum(axis=0)
    return F, J


def ff_forces(theta, cell, pos, rc):
    """F_i = -dE/dR_i of E = 1/2 sum_{i, j, L}' phi_s(|R_j + L - R_i|), where phi_s is phi
    shifted so that phi_s(rc) = phi_s'(rc) = 0 (shifted force) and zero beyond rc."""
    pos = np.asarray(pos, float)
    n = len(pos)
    Ls = image_vectors(cell, rc)
    dc = morse_dphi(theta, rc)
    F = np.zeros((n, 3))
    for i in range(n):
        for j in range(n):
            rv = pos[j][None, :] + Ls - pos[i][None, :]
            r = np.linalg.norm(rv, axis=1)
            m = (r < rc) & (r > 1e-12)
            if i == j:
                continue  # an atom's own images do not move with it relative to itself
            rr = r[m]
            dphi = morse_dphi(theta, rr) - dc
            F[i] += ((dphi / rr)[:, None] * rv[m]).sum(axis=0)
    return F


REG = 1e-6          # weight of the pull towards the previous parameters, per force component


def fit_force_field(history, theta0, cell, rc, iters=60, reg=REG):
    """Levenberg-Marquardt fit of theta = (D, a, r0) to every (positions, DFT forces) pair
    in history: minimise sum |F_ff(theta; x) - F_dft|^2 + w sum_k ((theta_k - theta0_k) /
    theta0_k)^2, w = reg * mean(F_dft^2) * (number of force components): a few forces
    (a dimer has one number) leave the three parameters undetermined, and the small pull
    towards the previous fit picks the nearest solution.  The Jacobian of the force
    residual is analytic (ff_forces_jac).  Returns theta0 unchanged if the fit leaves
    D, a, r0 > 0 or turns non-finite."""
    theta = np.array(theta0, float)
    t0 = np.array(theta0, float)
    fall = np.concatenate([f.ravel() for _, f in history])
    sw = np.sqrt(reg * max(np.mean(fall * fall), 1e-30) * len(fall))

    def resid(t):
        return np.concatenate([(ff_forces(t, cell, x, rc) - f).ravel() for x, f in history] +
                              [sw * (t - t0) / t0])

    def jac(t):
        rows = [ff_forces_jac(t, cell, x, rc)[1].reshape(-1, 3) for x, _ in history]
        return np.concatenate(rows + [np.diag(sw / t0)])

    r = resid(theta)
    cost = r @ r
    lam = 1e-3
    for _ in range(iters):
        J = jac(theta)
        A = J.T @ J
        g = J.T @ r
        improved = False
        while lam < 1e12:
            step = np.linalg.solve(A + lam * np.diag(np.diag(A) + 1e-30), -g)
            t = theta + step
            if np.all(t > 0):
                rn = resid(t)
                cn = rn @ rn
                if np.isfinite(cn) and cn < cost:
                    theta, r, cost = t, rn, cn
                    lam = max(lam / 10.0, 1e-12)
                    improved = True
                    break
            lam *= 10.0
        if not improved or np.abs(step).max() <= 1e-10 * np.abs(theta).max():
            break
    if not (np.all(np.isfinite(theta)) and np.all(theta > 0)):
        return np.array(theta0, float)
    return theta


def ff_hessian(theta, cell, pos, rc, h=H_FD):
    """H = second-order finite difference of the fitted energy: column k is
    -(F(x + h e_k) - F(x - h e_k)) / 2h, then symmetrised."""
    pos = np.asarray(pos, float)
    n3 = pos.size
    H = np.empty((n3, n3))
    for k in range(n3):
        xp, xm = pos.copy().ravel(), pos.copy().ravel()
        xp[k] += h
        xm[k] -= h
        H[:, k] = -(ff_forces(theta, cell, xp.reshape(-1, 3), rc) - ff_forces(theta, cell, xm.reshape(-1, 3), rc)).ravel() / (2 * h)
    return 0.5 * (H + H.T)


def truncated_inverse(H, floor=FLOOR):
    """H^-1 = sum_j V_j V_j^T / tau_j over the eigenpairs of H except the three of smallest
    |tau| (the translations); |tau_j| is used, floored at floor * max|tau| (a positive
    definite preconditioner on the non-translational subspace)."""
    tau, V = np.linalg.eigh(H)
    order = np.argsort(np.abs(tau))
    keep = order[3:]
    t = np.abs(tau[keep])
    t = np.maximum(t, floor * t.max()) if len(t) else t
    Vk = V[:, keep]
    return (Vk / t) @ Vk.T


def nearest_neighbour(cell, pos):
    Ls = image_vectors(cell, 1.0)
    best = np.inf
    for i in range(len(pos)):
        for j in range(len(pos)):
            rv = pos[j][None, :] + Ls - pos[i][None, :]
            r = np.linalg.norm(rv, axis=1)
            r = r[r > 1e-9]
            if len(r):
                best = min(best, r.min())
    return best


# ---------------------------------------------------------------------------
# drivers
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Trajectory:
    positions: List[np.ndarray]      # every evaluated configuration, in order
    energies: List[float]
    forces: List[np.ndarray]
    converged: bool

    @property
    def final(self):
        return self.positions[-1]


def _fmax(F):
    return np.linalg.norm(F, axis=1).max()


def relax(ef: Callable[[np.ndarray], Tuple[float, np.ndarray]], cell, pos0, method="pcg", fmax=1e-3,
          max_evals=60, max_step=0.3, refit=3, rc=8.0, precond=None, accept=0.1):
    """Relax pos0 (natoms x 3, bohr) on the energy/force function ef(pos) -> (E, F).

    Nonlinear (P)CG, Polak-Ribiere+ with restarts: s = P g (g = -F), d = -s + beta d_prev,
    beta = max(0, g.(s - s_prev) / g_prev.s_prev), reset to -s when d.g >= 0.  Line
    minimisation along d from the directional derivatives (-F.d) at 0 and at a trial step
    a_t = min(a_prev, max_step / max_i |d_i|), a_prev the previous line's a* (1 at the
    start and whenever the preconditioner is renewed: a well-scaled preconditioner makes a*
    about 1, and a badly scaled one, such as a force field fitted too soft, is corrected
    after one line): secant a* = a_t p0 / (p0 - p_t) when the
    curvature is positive, else the largest step; a* is kept at >= 0.1 a_t and at most
    max_step of displacement from the start of the line; the trial point is kept as the
    new point when |a* - a_t| <= accept a_t (one evaluation saved; accept = 0 keeps every
    line minimisation exact on a quadratic).
    PCG preconditioner: the fitted force field's truncated inverse Hessian (renewed
    every `refit` directions; precond overrides it with a fixed matrix); CG: I / KAPPA0.
    BFGS: dx = -B g capped to max_step per atom, inverse update when s.y > 0, B0 = I / KAPPA0.
    Converged when max_i |F_i| < fmax at an evaluated point."""
    cell = np.asarray(cell, float)
    x = np.array(pos0, float)
    n3 = x.size
    traj = Trajectory([], [], [], False)

    def evaluate(p):
        E, F = ef(p)
        F = np.asarray(F, float).reshape(-1, 3)
        traj.positions.append(p.copy())
        traj.energies.append(float(E))
        traj.forces.append(F.copy())
        return F

    F = evaluate(x)
    if _fmax(F) < fmax:
        traj.converged = True
        return traj
    g = -F.ravel()
    if method == "bfgs":
        B = np.eye(n3) / KAPPA0
        while len(traj.positions) < max_evals:
            dx = -(B @ g)
            m = np.linalg.norm(dx.reshape(-1, 3), axis=1).max()
            if m > max_step:
                dx *= max_step / m
            xn = x + dx.reshape(-1, 3)
            Fn = evaluate(xn)
            gn = -Fn.ravel()
            if _fmax(Fn) < fmax:
                traj.converged = True
                return traj
            y = gn - g
            sy = dx @ y
            if sy > 1e-12:
                rho = 1.0 / sy
                I = np.eye(n3)
                B = (I - rho * np.outer(dx, y)) @ B @ (I - rho * np.outer(y, dx)) + rho * np.outer(dx, dx)
            x, g = xn, gn
        return traj

    theta = None
    P = None
    ndir = 0
    a_prev = 1.0      # the previous line's minimising step: the next trial step
    d_prev = s_prev = g_prev = None
    hist = [(x.copy(), F.copy())]
    while len(traj.positions) < max_evals:
        if method == "pcg":
            if precond is not None:
                P = precond
            elif P is None or ndir % refit == 0:
                if theta is None:
                    theta = np.array([0.1, 1.0, nearest_neighbour(cell, x)])
                theta = fit_force_field(hist[-HIST:], theta, cell, rc)
                P = truncated_inverse(ff_hessian(theta, cell, x, rc))
                a_prev = 1.0  # a step found under the previous preconditioner has its scale
        else:
            P = np.eye(n3) / KAPPA0
        s = P @ g
        if d_prev is None:
            d = -s
        else:
            beta = max(0.0, g @ (s - s_prev) / (g_prev @ s_prev))
            d = -s + beta * d_prev
            if d @ g >= 0:
                d = -s
        ndir += 1
        dmax = np.linalg.norm(d.reshape(-1, 3), axis=1).max()
        if dmax <= 0:
            break
        at = min(a_prev, max_step / dmax)
        xt = x + at * d.reshape(-1, 3)
        Ft = evaluate(xt)
        hist.append((xt.copy(), Ft.copy()))
        if _fmax(Ft) < fmax:
            traj.converged = True
            return traj
        gt = -Ft.ravel()
        p0, pt = g @ d, gt @ d
        amax = max_step / dmax
        a_star = at * p0 / (p0 - pt) if pt - p0 > 0 else amax  # zero of the secant of phi'
        a_star = min(max(a_star, 0.1 * at), amax)
        a_prev = a_star
        g_prev, s_prev, d_prev = g, s, d
        if abs(a_star - at) <= accept * at or len(traj.positions) >= max_evals:
            x, g = xt, gt
            continue
        x = x + a_star * d.reshape(-1, 3)
        Fn = evaluate(x)
        hist.append((x.copy(), Fn.copy()))
        if _fmax(Fn) < fmax:
            traj.converged = True
            return traj
        g = -Fn.ravel()
    return traj
