"""Seeded synthetic specimens shared, as input data only, by the CUDA path and the oracle."""
from .mesh import (Workload, HexWorkload, hex_block, kuhn_block, plate_small, plate_medium, plate_large, union, ensemble, ensemble_members,
                   adjoint_block, top_face_weights,
                   scaled_plate, splitmix64, uniform01, normal01, lognormal)
