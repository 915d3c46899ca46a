"""GB300 (sm_103a) engine for the DPD-CGMD multiscale blood-clot model with
multiple time stepping (arXiv 2205.14121).

The compute path is ``libmsm.so`` (hand-written CUDA, C ABI in
``include/msm.h``); this package only marshals arguments to it
(:mod:`._binding`) and uses PyTorch for the device workspace and the stream.
Importing works without a GPU; creating a :class:`System` needs one and fails
loudly when the library has not been built.
"""
from ._binding import (  # noqa: F401
    MD_LEVEL_ALL, MD_LEVEL_FLUID, MD_LEVEL_IFACE, MD_LEVEL_PLT, MD_LIST_FLUID, MD_LIST_IFACE, MD_LIST_LJ,
    MD_LIST_MORSE, MD_CFG_UNIFORM_NOISE, MD_CFG_LEES_EDWARDS, MD_CFG_WALLS, MD_MODE_RESPA, MD_MODE_STS, MD_MODE_AI,
    MD_SCHED_DETERMINISTIC, RECEPTOR_BIT, MdError, System, config_for, lib, library_path,
)
