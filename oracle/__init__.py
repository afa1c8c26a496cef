"""CPU FP64 oracle of the CEM step.  Test infrastructure only: imported by tests,
the smoke check and the CPU-baseline leg of the benchmark, never by the product path."""
from .cem_oracle import (CEMOracle, lame, elasticity_matrix, tet_geometry, strain_matrix,
                         principal_stress_projection, sub_tet_nodes, crack_area,
                         normalize_side, pattern_of_side, LOCAL_EDGES, LOCAL_FACES,
                         PATTERN_I, PATTERN_II, voigt_to_tensor)
from .hex_oracle import (HexOracle, HEX_EDGES, HEX_FACES, HEX_XI, hex_volume, hex_edge_gradients,  # noqa: E402
                         hex_strain_matrix)
