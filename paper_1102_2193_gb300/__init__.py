"""GB300-native hybrid lattice Boltzmann / Beris-Edwards solver for colloids in liquid crystals.

The compute path is the CUDA library ``liblclb.so`` (sm_103a) behind the C ABI
declared in ``include/lc_lb.h``; this package is its thin Python binding
(argument marshalling only).  Importing the package does not load the
library; :func:`lib` does, and raises if it has not been built.
"""
from __future__ import annotations

import math

from ._binding import (  # noqa: F401
    LC_FP32, LC_FP64, LC_NORMAL, LC_PLANAR, LC_Q, LC_U, LC_RHO, LC_F_PRE, LC_FORCE, LcLbError, Solver, Batch, lib,
    library_path, LC_OK, LC_ERR_ARG, LC_ERR_CUDA, LC_ERR_OOM, LC_ERR_OVERLAP, LC_ERR_NONFINITE, LC_ERR_TIMEOUT,
    LC_ERR_STATE,
)


def dimensionless(A0: float, K: float, gamma: float, q0: float, Gamma: float, q: float, v: float = 0.0,
                  R: float = 0.0) -> dict:
    """Dimensionless groups of Sec. 2.1 (Eqs. 5-6).

    chirality kappa = sqrt(108 K q0^2 / (A0 gamma)), reduced temperature
    tau = 27 (1 - gamma/3)/gamma, rotational viscosity gamma_1 = 2 q^2 / Gamma
    and the Ericksen number Er = gamma_1 v R / K.
    """
    g1 = 2.0 * q * q / Gamma
    return dict(kappa=math.sqrt(108.0 * K * q0 * q0 / (A0 * gamma)), tau=27.0 * (1.0 - gamma / 3.0) / gamma,
                gamma1=g1, Er=g1 * v * R / K if K else float("inf"))


def bulk_order(gamma: float) -> float:
    """Uniaxial order parameter that minimises the bulk part of Eq. 1."""
    t = 1.0 - 8.0 / (3.0 * gamma)
    return 0.25 + 0.75 * math.sqrt(t) if t >= 0 else 0.0
