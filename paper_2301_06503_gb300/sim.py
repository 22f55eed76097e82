"""Python handle over one LGDM simulation in the CUDA library.

``Sim`` marshals a mesh, material and Dirichlet list (any objects with the
attribute names of ``lgdm_inputs``), takes its device workspace from
PyTorch's allocator and its stream from PyTorch's current stream, and
forwards every step to the C ABI.  All arithmetic of the method runs in the
library's kernels.
"""
import ctypes as C

import numpy as np
import torch

from . import _lib as L

_PREC = {"fp64": L.PREC_FP64, "fp32": L.PREC_FP32_TANGENT, "fp32_tangent": L.PREC_FP32_TANGENT}
_PRECOND = {"jacobi": L.PRECOND_JACOBI, "block": L.PRECOND_NODE_BLOCK, "multigrid": L.PRECOND_MULTIGRID}


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


def _p(a, ct):
    return None if a is None else a.ctypes.data_as(C.POINTER(ct))


def make_options(precision="fp64", precond="multigrid", newton_tol=1e-8, krylov_rtol=None, max_newton=50,
                 max_krylov=5000, max_halvings=6, krylov_blocks=0, gmres_m=64, krylov="bicgstab",
                 wait_limit_s=2.0):
    o = L.Options()
    L.check(L.load().lgdm_default_options(C.byref(o)))
    o.precision = _PREC[precision]
    o.precond = _PRECOND[precond]
    o.newton_tol = newton_tol
    o.krylov_rtol = krylov_rtol if krylov_rtol is not None else (1e-6 if o.precision else 1e-9)
    o.max_newton = max_newton
    o.max_krylov = max_krylov
    o.max_halvings = max_halvings
    o.krylov_blocks = krylov_blocks
    o.gmres_m = gmres_m
    o.krylov_method = {"bicgstab": 0, "gmres": 1}[krylov]
    o.wait_limit_s = wait_limit_s
    return o


class _MeshArgs:
    """ctypes mesh struct plus the numpy arrays it points into."""

    def __init__(self, mesh):
        self.arrs = [_f64(mesh.x), _f64(mesh.y) if mesh.y is not None else None,
                     _f64(mesh.z) if mesh.z is not None else None, _i32(mesh.conn).ravel(),
                     _f64(mesh.e_scale), _f64(mesh.vol_scale)]
        x, y, z, conn, es, vs = self.arrs
        self.s = L.Mesh(int(mesh.elem), int(x.shape[0]), int(conn.shape[0] // L.NEN[int(mesh.elem)]),
                        _p(x, C.c_double), _p(y, C.c_double), _p(z, C.c_double), _p(conn, C.c_int32),
                        _p(es, C.c_double), _p(vs, C.c_double))


def pattern_counts(mesh):
    """(node pairs, CSR nonzeros) of the mesh's fixed pattern; host only."""
    m = _MeshArgs(mesh)
    npairs, nnz = C.c_int64(), C.c_int64()
    L.check(L.load().lgdm_pattern_counts(C.byref(m.s), C.byref(npairs), C.byref(nnz)))
    return int(npairs.value), int(nnz.value)


def workspace_bytes(mesh, **opts) -> int:
    m = _MeshArgs(mesh)
    n = C.c_size_t()
    L.check(L.load().lgdm_workspace_size(C.byref(m.s), C.byref(make_options(**opts)), C.byref(n)))
    return int(n.value)


class Sim:
    def __init__(self, mesh, material, bcs, device=None, stream=None, fill_workspace=None, **opts):
        lib = L.load()
        self._lib = lib
        self.h = None
        m = _MeshArgs(mesh)
        mat = L.Material(*[float(getattr(material, n)) for n in
                           ("E", "nu", "k", "kappa0", "alpha", "beta", "R", "eta", "c", "h")],
                         int(getattr(material, "evm_variant", 0)), int(getattr(material, "h_stress", 0)))
        dof, scale = _i32(bcs.dir_dof), _f64(bcs.dir_scale)
        b = L.BCs(int(dof.shape[0]), _p(dof, C.c_int32), _p(scale, C.c_double))
        self.options = make_options(**opts)
        n = C.c_size_t()
        L.check(lib.lgdm_workspace_size(C.byref(m.s), C.byref(self.options), C.byref(n)))
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.workspace = torch.empty(int(n.value), dtype=torch.uint8, device=self.device)
        if fill_workspace is not None:                 # debugging aid: poison the workspace
            self.workspace.fill_(int(fill_workspace))
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            L.check(lib.lgdm_create(C.byref(m.s), C.byref(mat), C.byref(b), C.byref(self.options),
                                    C.c_void_p(self.workspace.data_ptr()), int(n.value),
                                    C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h
        sz = L.Sizes()
        L.check(lib.lgdm_get_sizes(h, C.byref(sz)))
        self.sizes = sz
        self.ndof, self.nnz, self.nel, self.ngp = int(sz.ndof), int(sz.nnz), int(sz.nelem), int(sz.ngp)
        self.nd, self.dim = int(sz.nd), int(sz.dim)

    # -------------------------------------------------------------- lifecycle
    def close(self):
        if self.h is not None:
            torch.cuda.synchronize(self.device)
            self._lib.lgdm_destroy(self.h)
            self.h = None
            self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, st):
        L.check(st, self.h)

    # -------------------------------------------------------------- state
    def set_state(self, u=None, kappa_hist=None):
        u = _f64(u)
        k = _f64(kappa_hist)
        if u is not None and u.shape != (self.ndof,):
            raise ValueError("u must have ndof entries")
        if k is not None and k.shape != (self.nel * self.ngp,):
            raise ValueError("kappa_hist must have nelem*ngp entries")
        self._ck(self._lib.lgdm_set_state(self.h, _p(u, C.c_double), _p(k, C.c_double)))

    def reset_state(self):
        """Back to u = 0, kappa_hist = kappa0 on the device (no re-creation)."""
        self._ck(self._lib.lgdm_reset_state(self.h))

    def field(self, which) -> np.ndarray:
        """A field copied to the host: "u" (interleaved dofs), "displacement"
        (nodes x dim), "ebar" (nodal micro-equivalent strain), "kappa_hist" and
        "damage" (per Gauss point, element-major), "delta", "residual", "rhs"."""
        if which in ("displacement", "ebar"):
            u = self.field("u").reshape(-1, self.nd)
            return u[:, :self.dim].copy() if which == "displacement" else u[:, self.dim].copy()
        which = {"u": L.FIELD_U, "kappa_hist": L.FIELD_KAPPA_HIST, "damage": L.FIELD_DAMAGE,
                 "delta": L.FIELD_DELTA, "residual": L.FIELD_RESIDUAL, "rhs": L.FIELD_RHS}.get(which, which)
        n = self.nel * self.ngp if which in (L.FIELD_KAPPA_HIST, L.FIELD_DAMAGE) else self.ndof
        out = np.empty(n)
        self._ck(self._lib.lgdm_get_field(self.h, int(which), _p(out, C.c_double), n))
        return out

    # -------------------------------------------------------------- method steps
    def begin_step(self, load):
        self._ck(self._lib.lgdm_begin_step(self.h, float(load)))

    def assemble(self):
        self._ck(self._lib.lgdm_assemble(self.h))

    def system(self):
        """Assembled (rowptr, col, vals, rhs) as numpy arrays (vals in float64)."""
        rp = np.empty(self.ndof + 1, np.int32)
        col = np.empty(self.nnz, np.int32)
        vals = np.empty(self.nnz)
        rhs = np.empty(self.ndof)
        self._ck(self._lib.lgdm_get_system(self.h, _p(rp, C.c_int32), _p(col, C.c_int32),
                                           _p(vals, C.c_double), _p(rhs, C.c_double)))
        return rp, col, vals, rhs

    def solve(self):
        it, rel = C.c_int32(), C.c_double()
        self._ck(self._lib.lgdm_solve(self.h, C.byref(it), C.byref(rel)))
        return int(it.value), float(rel.value)

    def update(self):
        cv = C.c_int32()
        self._ck(self._lib.lgdm_update(self.h, C.byref(cv)))
        return bool(cv.value)

    def newton_step(self):
        cv, it = C.c_int32(), C.c_int32()
        self._ck(self._lib.lgdm_newton_step(self.h, C.byref(cv), C.byref(it)))
        return bool(cv.value), int(it.value)

    def run_step(self, load):
        it = C.c_int32()
        self._ck(self._lib.lgdm_run_step(self.h, float(load), C.byref(it)))
        return int(it.value)

    def commit(self):
        self._ck(self._lib.lgdm_commit(self.h))

    def last_solve(self):
        """(krylov iterations, status, relative residual, [|du|, |u|, |de|, |e|]) of the last launch."""
        it, st, rel = C.c_int32(), C.c_int32(), C.c_double()
        nrm = np.zeros(4)
        self._ck(self._lib.lgdm_last_solve(self.h, C.byref(it), C.byref(st), C.byref(rel), _p(nrm, C.c_double)))
        return int(it.value), int(st.value), float(rel.value), nrm

    def enable_timers(self, on=True):
        self._ck(self._lib.lgdm_enable_timers(self.h, 1 if on else 0))

    def timers(self, reset=False):
        """{phase: (milliseconds, launches)} from the CUDA-event phase timers."""
        ms = np.zeros(L.NPHASES)
        n = np.zeros(L.NPHASES, np.int64)
        self._ck(self._lib.lgdm_get_timers(self.h, _p(ms, C.c_double), _p(n, C.c_int64)))
        if reset:
            self._ck(self._lib.lgdm_reset_timers(self.h))
        return {name: (float(ms[k]), int(n[k])) for k, name in enumerate(L.PHASES)}

    def counters(self):
        c = np.zeros(len(L.COUNTERS), np.int64)
        self._ck(self._lib.lgdm_get_counters(self.h, _p(c, C.c_int64), len(L.COUNTERS)))
        return {name: int(c[k]) for k, name in enumerate(L.COUNTERS)}

    def reaction(self) -> float:
        r = C.c_double()
        self._ck(self._lib.lgdm_get_reaction(self.h, C.byref(r)))
        return float(r.value)

    def energy(self) -> float:
        """Stored energy (Eq. 1) at the current state."""
        e = C.c_double()
        self._ck(self._lib.lgdm_get_energy(self.h, C.byref(e)))
        return float(e.value)

    def committed(self):
        """(load, external work, reaction) of the committed state."""
        ld, w, r = C.c_double(), C.c_double(), C.c_double()
        self._ck(self._lib.lgdm_get_committed(self.h, C.byref(ld), C.byref(w), C.byref(r)))
        return float(ld.value), float(w.value), float(r.value)

    def set_committed(self, load, external_work, reaction):
        self._ck(self._lib.lgdm_set_committed(self.h, float(load), float(external_work), float(reaction)))

    def checkpoint(self) -> dict:
        """Everything a resumed run needs: dofs, history and committed scalars."""
        load, w, r = self.committed()
        return {"u": self.field("u"), "kappa_hist": self.field("kappa_hist"), "load": load,
                "external_work": w, "reaction": r}

    def restore(self, ck):
        self.set_state(ck["u"], ck["kappa_hist"])
        self.set_committed(ck["load"], ck["external_work"], ck["reaction"])

    def dissipated_energy(self):
        """(dissipated energy, stored energy) at the committed state."""
        d, e = C.c_double(), C.c_double()
        self._ck(self._lib.lgdm_get_dissipated_energy(self.h, C.byref(d), C.byref(e)))
        return float(d.value), float(e.value)

    def damaged_volume(self, threshold=0.9) -> float:
        """Volume of the Gauss points whose committed damage exceeds threshold."""
        v = C.c_double()
        self._ck(self._lib.lgdm_get_damaged_volume(self.h, float(threshold), C.byref(v)))
        return float(v.value)

    def inject_fault(self, kind):
        """Failure injection for tests: 1 barrier timeout, 2 NaN state, 0 none."""
        self._ck(self._lib.lgdm_inject_fault(self.h, int(kind)))

    def snapshot(self, path=None) -> dict:
        """Fields of the committed state, headless: damage and history per Gauss
        point, nodal displacement and micro-equivalent strain, with the load,
        reaction and damaged (D > 0.9) volume; written to ``path`` (.npz) if given."""
        load, w, r = self.committed()
        snap = {"load": load, "reaction": r, "external_work": w, "damage": self.field("damage"),
                "kappa_hist": self.field("kappa_hist"), "displacement": self.field("displacement"),
                "ebar": self.field("ebar"), "damaged_volume_0.9": self.damaged_volume(0.9)}
        if path is not None:
            np.savez(path, **snap)
        return snap

    def run(self, loads, snapshot_at=(), snapshot_dir=None):
        """Run the given load values in order; returns (reactions, newton_iters).
        After each load in ``snapshot_at`` the committed fields are stored
        (``self.snapshots[load]``, and snapshot_dir/snapshot_<load>.npz)."""
        reac, its = [], []
        marks = {float(x) for x in snapshot_at}
        self.snapshots = getattr(self, "snapshots", {})
        for lv in loads:
            its.append(self.run_step(lv))
            reac.append(self.reaction())
            if float(lv) in marks:
                path = None
                if snapshot_dir is not None:
                    import os
                    path = os.path.join(snapshot_dir, f"snapshot_{float(lv):.6g}.npz")
                self.snapshots[float(lv)] = self.snapshot(path)
        return np.asarray(reac), np.asarray(its)
