"""Seeded synthetic inputs (images, displacement fields, random vectors).

Shared by the tests, the benchmark and the examples; holds none of the
registration method's arithmetic.
"""
from .configs import CONFIGS, seed_for, batch_sizes  # noqa: F401
from .phantoms import (make_pair, make_pair_parallel, random_image, random_field, random_vector,  # noqa: F401
                       voxel_centres, true_inverse_displacement)
