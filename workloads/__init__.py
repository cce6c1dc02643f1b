"""Seeded synthetic inputs for the error-injecting state-vector simulator.

This package builds circuits (gate records), error angles and input states
from fixed seeds.  Both the CUDA path and the CPU oracle take their inputs
from here; the package holds none of the simulator's arithmetic (no gate is
ever applied to a state vector here, no fidelity or norm is computed).

The gate set follows Section 2.0 of the paper (one-, two- and three-bit
controlled-NOT gates plus rotation gates); operational errors are deviations
of rotation angles (Sections 1.4 and 2.0).  The exact conventions used where
the paper is silent are listed in the module docstring of
``workloads.generators``.
"""

from .generators import (  # noqa: F401
    GATE_DTYPE,
    gate_record,
    mat_h, mat_x, mat_rx, mat_ry, mat_rz, mat_phase, mat_haar_su2, su2_axis,
    mat_rot_axis,
    random_state,
    circuit_c1_random, circuit_c2_qft, circuit_brickwork, circuit_c4_brickwork_toffoli,
    trajectory_eps, serving_requests, inverse_circuit, records_to_arrays,
)
