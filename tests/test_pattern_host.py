"""The fixed CSR pattern and the workspace size, on the host (no GPU).

The node-pair count of a structured n_x x n_y (x n_z) element grid has a
closed form: along each axis a node sees itself and its neighbours within
one element, which sums to 3(n+1) - 2 over the axis, and the pattern is the
product over the axes; the CSR holds nd^2 values per pair.  Unstructured
numberings are checked against a brute-force set of node pairs that share an
element.  Invalid meshes are refused with LGDM_ERR_INVALID_ARG.
"""
import numpy as np
import pytest

import lgdm_inputs as li
from paper_2301_06503_gb300 import _lib, build


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _closed_form(ns):
    return int(np.prod([3 * (n + 1) - 2 for n in ns]))


@pytest.mark.parametrize("mesh, ns", [
    (lambda: li.bar_problem().mesh, (100,)),
    (lambda: li.sen_plate_problem(13, 7).mesh, (13, 7)),
    (lambda: li.sen_plate_problem().mesh, (200, 200)),
    (lambda: li.tpb_beam_problem(6, 5, 4, 6.0, 5.0, 4.0).mesh, (6, 5, 4)),
])
def test_structured_pattern_closed_form(mesh, ns):
    from paper_2301_06503_gb300.sim import pattern_counts
    m = mesh()
    npairs, nnz = pattern_counts(m)
    assert npairs == _closed_form(ns)
    assert nnz == m.nd * m.nd * npairs


def test_plate_pattern_matches_the_benchmark_table():
    """200 x 200 plate: 361,201 node pairs, 3,250,809 nonzeros."""
    from paper_2301_06503_gb300.sim import pattern_counts
    assert pattern_counts(li.sen_plate_problem().mesh) == (361201, 3250809)


def _brute_pairs(conn):
    pairs = set()
    for e in conn:
        for a in e:
            for b in e:
                pairs.add((int(a), int(b)))
    return len(pairs)


def test_permuted_numbering_against_brute_force():
    from paper_2301_06503_gb300.sim import pattern_counts
    m = li.tpb_beam_problem(4, 3, 3, 4.0, 3.0, 3.0).mesh
    rng = np.random.default_rng(0)
    perm = rng.permutation(m.nnode)                 # new id of every node
    inv = np.argsort(perm)
    m.conn = perm[m.conn]
    m.x, m.y, m.z = m.x[inv], m.y[inv], m.z[inv]
    npairs, nnz = pattern_counts(m)
    assert npairs == _brute_pairs(m.conn) == _closed_form((4, 3, 3))
    assert nnz == 16 * npairs


def test_invalid_meshes_are_refused():
    from paper_2301_06503_gb300.sim import pattern_counts
    m = li.sen_plate_problem(4, 4).mesh
    m.conn = m.conn.copy()
    m.conn[3, 2] = m.nnode                          # out of range
    with pytest.raises(_lib.LgdmError) as ei:
        pattern_counts(m)
    assert ei.value.status == 1                     # LGDM_ERR_INVALID_ARG
    assert "out of range" in str(ei.value)
    m2 = li.sen_plate_problem(4, 4).mesh
    m2.elem = 7                                     # unknown element type
    with pytest.raises((_lib.LgdmError, KeyError)):
        pattern_counts(m2)


def test_workspace_size_grows_with_the_mesh_and_shrinks_with_fp32():
    from paper_2301_06503_gb300.sim import workspace_bytes
    small = workspace_bytes(li.sen_plate_problem(20, 20).mesh)
    big = workspace_bytes(li.sen_plate_problem(40, 40).mesh)
    big32 = workspace_bytes(li.sen_plate_problem(40, 40).mesh, precision="fp32")
    assert 0 < small < big and big32 < big


def test_empty_and_degenerate_meshes():
    """An empty mesh, and one with a node that belongs to no element (its
    rows would be empty), are refused before any device work; a single
    element sizes correctly."""
    import copy
    from paper_2301_06503_gb300.sim import pattern_counts, workspace_bytes
    m = copy.deepcopy(li.sen_plate_problem(3, 3).mesh)
    m.conn = m.conn[:0]                              # no elements
    with pytest.raises(_lib.LgdmError) as ei:
        workspace_bytes(m)
    assert ei.value.status == 1
    one = li.sen_plate_problem(1, 1).mesh            # a single Q4
    assert pattern_counts(one) == (16, 16 * 9)
    spare = copy.deepcopy(li.sen_plate_problem(2, 2).mesh)
    spare.conn = spare.conn[:1]                      # one element of a 3 x 3 node grid: 5 nodes unused
    with pytest.raises(_lib.LgdmError) as ei:
        pattern_counts(spare)
    assert "belongs to no element" in str(ei.value)


@pytest.mark.parametrize("mesh", [lambda: li.bar_problem(n=7, order=2).mesh,
                                  lambda: li.sen_plate_problem(5, 4, order=2).mesh])
def test_mixed_order_pattern_against_brute_force(mesh):
    """3-node bars and 9-node quads: every node pair sharing an element,
    mid-side and centre nodes included (their micro-strain dof is held)."""
    from paper_2301_06503_gb300.sim import pattern_counts
    m = mesh()
    npairs, nnz = pattern_counts(m)
    assert npairs == _brute_pairs(m.conn)
    assert nnz == m.nd * m.nd * npairs
