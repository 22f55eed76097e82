"""Shared helpers for the GPU parity tests (oracle side and comparisons)."""
import numpy as np
import scipy.sparse as sp

from oracle import assembly as asm
from oracle import element as el


def oracle_system(mesh, mat, bcs, u, kh):
    """Oracle tangent with Dirichlet rows/columns and the matching right-hand side."""
    K, r = asm.assemble(mesh, mat, u, kh)
    Kb, rb = asm.apply_dirichlet(K, r, bcs.dir_dof)
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
