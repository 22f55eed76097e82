"""Seeded synthetic inputs for the localizing gradient damage method (LGDM).

This package builds the problems that both the CUDA path and the CPU oracle
consume: structured meshes (2- and 3-node bars, 4- and 9-node quadrilaterals,
8-node hexahedra), material parameter sets, Dirichlet boundary-condition lists,
random admissible states for parity checks, and request traces for the
serving loop.  It holds none of the method's arithmetic: no shape function,
no constitutive law, no assembly.  Every array is plain numpy (float64 or
int32) so it can be handed to either side unchanged.
"""
from .meshes import Mesh, bar_l2, bar_l3, plate_q4, plate_q9, beam_h8, node_dofs
from .problems import (
    Material, BCs, Problem, bar_problem, sen_plate_problem, tpb_beam_problem,
    paper_bar_problem, paper_sen_plate_problem, paper_sen_slab_problem,
    batch_plate_problems, serving_trace, random_state,
)

__all__ = [
    "Mesh", "bar_l2", "bar_l3", "plate_q4", "plate_q9", "beam_h8", "node_dofs",
    "Material", "BCs", "Problem", "bar_problem", "sen_plate_problem",
    "tpb_beam_problem", "paper_bar_problem", "paper_sen_plate_problem",
    "paper_sen_slab_problem", "batch_plate_problems", "serving_trace", "random_state",
]
