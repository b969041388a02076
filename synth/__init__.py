"""Seeded synthetic catalogs for the standard-siren likelihood.

This package only *produces inputs*: posterior-estimate (PE) samples, sky
pixels and their sky factors, galaxy catalogs, detected injections and walker
hyperpoints, with the shapes of the paper's O5-like workloads (Sec. 3).  It
holds none of the likelihood arithmetic: both the CPU oracle and the CUDA
library receive its arrays unchanged, and no expected value is derived from
anything computed here.
"""
from .catalog import (  # noqa: F401
    PARAM_NAMES,
    FIDUCIAL,
    PRIOR_BOX,
    make_catalog,
    make_hyperpoints,
    config_catalog,
    quantize_galaxies,
)
