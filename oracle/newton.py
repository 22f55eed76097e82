"""Incremental-iterative Newton driver (Algorithm 2), direct sparse solve.

Per load step n: the Dirichlet dofs take their prescribed values; then Newton
iterations assemble K and r at the current iterate, solve K delta = -r with
delta = 0 on Dirichlet dofs, update u and the micro-equivalent strain, and
stop when ||delta_u|| <= tol ||u|| and ||delta_e|| <= tol ||e|| (a zero
denominator falls back to an absolute 1e-30).  The history is committed only
after convergence: kappa_hist <- max(kappa_hist, ebar at the Gauss points)
(Eq. A.2).  When Newton does not converge within max_newton iterations the
increment is halved and retried from the committed state, at most
max_halvings times.
"""
from dataclasses import dataclass

import numpy as np
import scipy.sparse.linalg as spla

from . import assembly as asm
from . import constitutive as cm
from . import element as el


class NotConverged(RuntimeError):
    pass


@dataclass
class State:
    u: np.ndarray
    kappa_hist: np.ndarray
    load: float = 0.0


def initial_state(problem):
    mesh = problem.mesh
    return State(np.zeros(mesh.ndof), np.full(mesh.nel * mesh.ngp, problem.material.kappa0), 0.0)


def _split_norms(mesh, v):
    is_e = (np.arange(mesh.ndof) % mesh.nd) == mesh.dim
    return np.linalg.norm(v[~is_e]), np.linalg.norm(v[is_e])


def _rel_ok(dn, n, tol):
    return dn <= (tol * n if n > 0.0 else 1e-30)


def newton(problem, state, load):
    """Newton iterations for one load value from a committed state.

    Returns (u, iterations) on convergence, (None, iterations) otherwise.
    """
    mesh, mat, bcs = problem.mesh, problem.material, problem.bcs
    u = state.u.copy()
    u[bcs.dir_dof] = bcs.dir_scale * load
    for it in range(1, problem.max_newton + 1):
        K, r = asm.assemble(mesh, mat, u, state.kappa_hist)
        Kb, rb = asm.apply_dirichlet(K, r, bcs.dir_dof, mesh)
        du = spla.spsolve(Kb.tocsc(), -rb)
        if not np.all(np.isfinite(du)):
            return None, it
        u += du
        dnu, dne = _split_norms(mesh, du)
        nu, ne = _split_norms(mesh, u)
        if _rel_ok(dnu, nu, problem.newton_tol) and _rel_ok(dne, ne, problem.newton_tol):
            return u, it
    return None, problem.max_newton


def commit(problem, state, u, load):
    ebar = el.gp_ebar(problem.mesh, u).ravel()
    return State(u, np.maximum(state.kappa_hist, ebar), load)


def advance(problem, state, load_to, depth=0, iters=None):
    """Move the committed state to ``load_to``, halving on non-convergence."""
    iters = [] if iters is None else iters
    u, it = newton(problem, state, load_to)
    iters.append(it)
    if u is not None:
        return commit(problem, state, u, load_to), iters
    if depth >= problem.max_halvings:
        raise NotConverged(f"load {load_to}: no convergence after {depth} halvings")
    mid = 0.5 * (state.load + load_to)
    s1, _ = advance(problem, state, mid, depth + 1, iters)
    return advance(problem, s1, load_to, depth + 1, iters)


def reaction_at(problem, state):
    _, r = asm.assemble(problem.mesh, problem.material, state.u, state.kappa_hist,
                        with_tangent=False)
    return asm.reaction(r, problem.bcs)


def free_energy(problem, state, chunk=20000):
    """Stored energy: integral of Eq. 1 over the mesh at a state, with the
    trial history max(kappa_hist, ebar) (at a committed state: kappa_hist).
    A complex state (complex-step derivatives) gives a complex value."""
    mesh, mat = problem.mesh, problem.material
    total = 0.0
    for s in range(0, mesh.nel, chunk):
        elems = np.arange(s, min(s + chunk, mesh.nel))
        t = el.element_terms(mesh, mat, state.u, state.kappa_hist, elems)
        psi = cm.free_energy_density(t["D"], t["eps"], t["Ceps"], mat.h, t["eps_eq"],
                                     t["ebar"], t["g"], mat.c, t["gbar"])
        total = total + np.sum(psi * t["dV"])
    return float(total) if np.isrealobj(total) else complex(total)


def damaged_volume(problem, state, threshold):
    """Volume of the region whose committed damage D(kappa_hist) (Eq. A.1)
    exceeds ``threshold``: the sum of dV over those Gauss points."""
    mesh, mat = problem.mesh, problem.material
    _, dV = el.geometry(mesh, np.arange(mesh.nel))
    D, _ = cm.damage(state.kappa_hist, mat.kappa0, mat.alpha, mat.beta)
    return float(np.sum(dV.ravel()[D > threshold]))


def run(problem, n_steps=None, state=None, first_step=1, energy=True):
    """Run load steps first_step..n_steps; returns the curve and the final state."""
    n_steps = problem.n_steps if n_steps is None else n_steps
    state = initial_state(problem) if state is None else state
    loads, reactions, newton_iters, psi = [], [], [], []
    for n in range(first_step, n_steps + 1):
        state, its = advance(problem, state, problem.load(n))
        loads.append(state.load)
        reactions.append(reaction_at(problem, state))
        newton_iters.append(int(sum(its)))
        psi.append(free_energy(problem, state) if energy else np.nan)
    loads, reactions, psi = map(np.asarray, (loads, reactions, psi))
    out = dict(load=loads, reaction=reactions, newton_iters=np.asarray(newton_iters),
               psi=psi, state=state)
    if energy:
        lp = np.concatenate([[0.0], loads]) if first_step == 1 else loads
        rp = np.concatenate([[0.0], reactions]) if first_step == 1 else reactions
        w_ext = np.concatenate([[0.0], np.cumsum(0.5 * (rp[1:] + rp[:-1]) * np.diff(lp))])
        out["w_ext"] = w_ext[1:] if first_step == 1 else w_ext
        out["dissipated"] = out["w_ext"] - psi
    return out
