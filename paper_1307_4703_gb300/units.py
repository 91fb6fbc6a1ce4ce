"""Conversion between physical and lattice units (section "Choice of
Parameter Values and Conversion", Tables 1-3 of Tanaka & Iber).

Lattice quantities are measured in the lattice spacing dx and the time step
dt.  A physical length L is resolved by L / dx nodes; the time step follows
from matching the maximal fluid speed U in both unit systems
(U_lb = U dt / dx); the viscosity, diffusion coefficient and decay rate then
convert as nu dt / dx^2, D dt / dx^2 and k dt.  The relaxation times follow
from the lattice transport coefficients: nu = c_s^2 (tau_f - 1/2) with
c_s^2 = 1/3 for the D2Q9 fluid, and D = c_s^2 (tau_g - 1/2) for the scalar
lattice with rest weight w0, c_s^2 = (1 - w0) / 2 (the paper's D2Q4 lattice,
w0 = 0, gives D = (2 tau_g - 1) / 4).
"""
from dataclasses import dataclass


@dataclass(frozen=True)
class Conversion:
    dx: float  # lattice spacing, physical length units
    dt: float  # time step, physical time units

    @classmethod
    def from_resolution(cls, length, nodes, u_phys, u_lattice):
        """dx from resolving `length` by `nodes` lattice spacings, dt from
        matching the maximal speed u_phys to u_lattice."""
        dx = length / nodes
        return cls(dx, u_lattice * dx / u_phys)

    def velocity(self, u):
        return u * self.dt / self.dx

    def viscosity(self, nu):
        return nu * self.dt / self.dx ** 2

    def diffusivity(self, D):
        return D * self.dt / self.dx ** 2

    def rate(self, k):
        return k * self.dt

    def steps(self, T):
        return T / self.dt

    def length(self, L):
        return L / self.dx

    # lattice -> physical
    def velocity_phys(self, u_lb):
        return u_lb * self.dx / self.dt

    def time_phys(self, steps):
        return steps * self.dt


def tau_fluid(nu_lb):
    """Relaxation time of the D2Q9 fluid for a lattice viscosity."""
    return 3.0 * nu_lb + 0.5


def tau_scalar(D_lb, w0=0.0):
    """Relaxation time of the scalar lattice with rest weight w0 for a
    lattice diffusion coefficient (w0 = 0: the paper's D2Q4)."""
    return D_lb / ((1.0 - w0) / 2.0) + 0.5


def reynolds(L, U, nu):
    return L * U / nu


def peclet(L, U, D):
    return L * U / D


def rescale_velocity(u_lb, dt_from, dt_to):
    """A lattice velocity field computed with time step dt_from, expressed
    with time step dt_to (the stored fluid field read by the scalar solver
    with its larger time step)."""
    return u_lb * dt_to / dt_from
