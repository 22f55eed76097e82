"""Shared helpers for the GPU parity tests (oracle side and comparisons)."""
import numpy as np
import scipy.sparse as sp

from oracle import assembly as asm
from oracle import element as el


def oracle_system(mesh, mat, bcs, u, kh):
    """Oracle tangent with Dirichlet rows/columns and the matching right-hand side."""
    K, r = asm.assemble(mesh, mat, u, kh)
    Kb, rb = asm.apply_dirichlet(K, r, bcs.dir_dof, mesh)
    return Kb.tocsr(), -rb, r


def gpu_csr(sim):
    rp, col, vals, rhs = sim.system()
    K = sp.csr_matrix((vals, col, rp), shape=(sim.ndof, sim.ndof))
    return K, rhs


def block_errors(mesh, K, Kref):
    """max|K - Kref| / max|Kref| on each of the uu, ue, eu, ee blocks."""
    is_e = (np.arange(mesh.ndof) % mesh.nd) == mesh.dim
    D = (K - Kref).tocsr()
    out = {}
    for name, rm, cm in (("uu", ~is_e, ~is_e), ("ue", ~is_e, is_e), ("eu", is_e, ~is_e), ("ee", is_e, is_e)):
        ri, ci = np.nonzero(rm)[0], np.nonzero(cm)[0]
        ref = abs(Kref[ri][:, ci]).max()
        d = abs(D[ri][:, ci]).max()
        out[name] = d / ref if ref > 0 else d
    return out


def vector_errors(mesh, v, vref):
    is_e = (np.arange(mesh.ndof) % mesh.nd) == mesh.dim
    out = {}
    for name, m in (("u", ~is_e), ("e", is_e)):
        ref = np.abs(vref[m]).max()
        d = np.abs(v[m] - vref[m]).max()
        out[name] = d / ref if ref > 0 else d
    return out


def local_rows_oracle(mesh, mat, bcs, u, kh, nodes):
    """Oracle rows of the given nodes: assemble only their incident elements."""
    nodes = np.asarray(nodes)
    elems = np.nonzero(np.isin(mesh.conn, nodes).any(axis=1))[0]
    t = el.element_terms(mesh, mat, u, kh, elems)
    Ke, rl = el.element_matrix(t)
    gu, ge = el.local_dofs(mesh, elems)
    gl = np.concatenate([gu, ge], axis=1)
    rows = (mesh.nd * nodes[:, None] + np.arange(mesh.nd)[None, :]).ravel()
    pos = {int(r): i for i, r in enumerate(rows)}
    ndl = gl.shape[1]
    R, Cc, V = [], [], []
    r = np.zeros(len(rows))
    for e in range(len(elems)):
        for i in range(ndl):
            k = pos.get(int(gl[e, i]))
            if k is None:
                continue
            r[k] += rl[e, i]
            R.append(np.full(ndl, k))
            Cc.append(gl[e])
            V.append(Ke[e, i])
    K = sp.coo_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(Cc))),
                      shape=(len(rows), mesh.ndof)).tocsr()
    isdir = np.zeros(mesh.ndof, bool)
    isdir[bcs.dir_dof] = True
    isdir[el.unused_dofs(mesh)] = True
    K = K.tolil()
    for k, row in enumerate(rows):
        if isdir[row]:
            K[k, :] = 0
            K[k, row] = 1.0
    K = K.tocsr()
    colmask = sp.diags((~isdir).astype(float))
    K = (K @ colmask).tolil()
    for k, row in enumerate(rows):
        if isdir[row]:
            K[k, row] = 1.0
    rhs = np.where(isdir[rows], 0.0, -r)
    return rows, K.tocsr(), rhs


# Accuracy of each result against the FP64 oracle (peak load and dissipated
# energy relative, damage field absolute over all Gauss points): the FP64 path
# to curve parity, the FP32-tangent path (inexact Newton) to its own targets.
# Both sides stop Newton at increments of 1e-8 relative, so a converged
# micro-strain field carries errors of that order, and the damage slope
# dD/dkappa (up to ~1e4 here) turns them into damage differences of ~1e-8:
# the FP64 damage bound is 1e-7.
ACCURACY = {"fp64": {"curve": 1e-6, "peak": 1e-6, "dissipated": 1e-6, "damage": 1e-7},
            "fp32": {"curve": 1e-6, "peak": 1e-4, "dissipated": 1e-4, "damage": 1e-5}}


def accuracy(p, g, reac, psi, dmg, dissipated=None):
    """Errors of a GPU run against a stored oracle run.  The dissipated energy
    is the one the library reports (``dissipated``) or, if not given, the
    external work (trapezoid rule over the load-displacement points) minus the
    stored energy ``psi`` (Eq. 1) at the last committed state."""
    reac = np.asarray(reac)
    if dissipated is None:
        load = np.concatenate([[0.0], np.asarray(g["load"])])
        rp = np.concatenate([[0.0], reac])
        w_ext = float(np.sum(0.5 * (rp[1:] + rp[:-1]) * np.diff(load)))
        dissipated = w_ext - psi
    ref = np.asarray(g["reaction"])
    out = {"curve": np.abs(reac - ref).max() / np.abs(ref).max(),
           "peak": abs(reac.max() - ref.max()) / abs(ref.max()),
           "dissipated": abs(dissipated - g["dissipated"][-1]) / abs(g["dissipated"][-1])}
    if "damage_final" in g and dmg is not None:
        dref = np.zeros(g["damage_final"]["n_gp"])
        dref[np.asarray(g["damage_final"]["idx"], dtype=np.int64)] = g["damage_final"]["val"]
        out["damage"] = np.abs(dmg - dref).max()
    return out
