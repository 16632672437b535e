"""Permeability of a porous geometry from a body-force driven steady flow.

The flow is advanced in rounds of `check` steps; each round's first kernel
also reduces (FP64, fixed order) the flux sum(rho u_x) of the state the round
starts from.  Converged when |Phi_m - Phi_{m-1}| < tol |Phi_m| for two
consecutive rounds' fluxes; k is taken from Phi_m.  Darcy: k = nu <rho u_x> / g, the average taken
over every cell of the box (superficial velocity), nu = (1/omega - 1/2)/3.
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


def permeability(flux: float, cells: int, omega: float, gx: float) -> float:
    nu = (1.0 / omega - 0.5) / 3.0
    return nu * (flux / cells) / gx


def solve(lat, omega: float, gx: float, check: int = 100, tol: float = 1e-6,
          max_steps: int = 200000) -> Solve:
    """Run `lat` (a lbm.Lattice with its state initialised) to a steady flux."""
    if check % 2:
        raise ValueError("check interval must be even (AA pattern read-out)")
    cells = int(lat.info.cells)
    prev = None
    steps = 0
    mass = flux = 0.0
    while steps < max_steps:
        mass, flux = lat.step_flux(check)  # flux of the state this round starts from
        steps += check
        if prev is not None and abs(flux - prev) < tol * abs(flux):
            return Solve(permeability(flux, cells, omega, gx), flux, mass, steps, True)
        prev = flux
    return Solve(permeability(flux, cells, omega, gx), flux, mass, steps, False)
