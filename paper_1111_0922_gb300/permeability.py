"""Permeability of a porous geometry from a body-force driven steady flow.

The whole solve runs in the library (lbm_solve_permeability, include/lbm.h):
rounds of `check` steps, each round's first kernel reducing (FP64, fixed
order) the flux sum(rho u_x) of the state the round starts from; converged
when the fluxes of two consecutive rounds differ by less than tol times
their magnitude; Darcy's k = nu <rho u_x> / g with the average over every
cell of the box (superficial velocity), nu = (1/omega - 1/2)/3.  This module
only names the result.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass
class Solve:
    k: float
    flux: float
    mass: float
    steps: int
    converged: bool


def solve(lat, check: int = 100, tol: float = 1e-6, max_steps: int = 200000) -> Solve:
    """Run `lat` (a lbm.Lattice with its state initialised) to a steady flux."""
    k, mass, flux, steps, converged = lat.solve_permeability(check, tol, max_steps)
    return Solve(k, flux, mass, steps, converged)
