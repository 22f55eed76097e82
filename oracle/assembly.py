"""Global assembly, Dirichlet handling and reaction (Algorithm 1).

The element blocks are unrolled into (row, col, value) triplets and summed
into a sparse matrix, as the paper's ``sparse(row, col, val)`` assembly does;
scipy sums duplicate entries.  The residual is summed the same way.
"""
import numpy as np
import scipy.sparse as sp

from . import element as el


def assemble(mesh, mat, u, kappa_hist, chunk=20000, with_tangent=True):
    """Global tangent K (CSR, ndof x ndof) and residual r = -F (ndof)."""
    ndof = mesh.ndof
    r = np.zeros(ndof, dtype=np.result_type(np.asarray(u).dtype, float))
    rows, cols, vals = [], [], []
    for s in range(0, mesh.nel, chunk):
        elems = np.arange(s, min(s + chunk, mesh.nel))
        t = el.element_terms(mesh, mat, u, kappa_hist, elems)
        Ke, re_ = el.element_matrix(t)
        gu, ge = el.local_dofs(mesh, elems)
        gl = np.concatenate([gu, ge], axis=1)                     # (ne, ndl)
        np.add.at(r, gl.ravel(), re_.ravel())
        if with_tangent:
            ndl = gl.shape[1]
            rows.append(np.repeat(gl, ndl, axis=1).ravel())
            cols.append(np.tile(gl, (1, ndl)).ravel())
            vals.append(Ke.ravel())
    if not with_tangent:
        return None, r
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(ndof, ndof)).tocsr()
    K.sum_duplicates()
    return K, r


def apply_dirichlet(K, r, dir_dof, mesh=None):
    """Identity rows and zero columns on constrained dofs; zero right-hand side.

    Newton increments vanish on Dirichlet dofs because their prescribed values
    were already set at the start of the load step.  With ``mesh`` the
    micro-equivalent-strain dofs no element interpolates (mixed order) are
    held at zero the same way: their rows and columns are empty, so this is
    the same as leaving them out of the system.
    """
    m = np.ones(K.shape[0])
    m[dir_dof] = 0.0
    if mesh is not None:
        m[el.unused_dofs(mesh)] = 0.0
    M = sp.diags(m)
    Kb = (M @ K @ M + sp.diags(1.0 - m)).tocsr()
    return Kb, r * m


def reaction(r, bcs):
    """Generalized force conjugate to the load parameter: sum_i s_i r[dof_i]."""
    return float(np.sum(bcs.dir_scale * np.real(r[bcs.dir_dof])))
