"""Seeded synthetic workloads shared by the oracle and the GPU library.

This module only describes problems and draws their random numbers: mesh
sizes, element sizes, per-element Young's moduli, Poisson ratio, which face is
clamped, and the load description (a body force, random face pressures or
random nodal forces).  It contains none of the solver's arithmetic; each side
(the oracle and the CUDA library) assembles its own stiffness matrix and load
vector from this description.

The five recipes stand in for the paper's multi-million-dof structural
matrices (Sec. 4, Table realWorldProblems), which are not available: they are
structured Q1-hex meshes like the paper's only hexahedral case (beam6502k,
App. A.6: a clamped, multi-material cantilever), with material jumps, high
aspect ratios and random loads as the sources of ill-conditioning.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED = 20190205


@dataclass
class Problem:
    name: str
    nx: int
    ny: int
    nz: int
    hx: float
    hy: float
    hz: float
    nu: float
    E: np.ndarray                  # (nx*ny*nz,) Young's modulus per element
    clamp_axis: int                # 0: x = 0 face clamped, 2: z = 0 face clamped
    load: str                      # "body" | "top_pressure" | "end_shear" | "top_nodal" | "ones"
    body: tuple = (0.0, 0.0, -1.0)
    pressure: np.ndarray | None = None   # (nx*ny,) per top-face element, pushes -z
    shear_total: float = -1.0           # resultant in z on the x = nx*hx face
    nodal: np.ndarray | None = None      # (k, (nx+1)*(ny+1), 3) forces on top-face nodes
    rho: np.ndarray | None = None        # SIMP densities (adjoint recipe)
    nu_elem: np.ndarray | None = None    # per-element Poisson ratio (two-material beam)
    nrhs: int = 1
    extra: dict = field(default_factory=dict)

    @property
    def ne(self):
        return self.nx * self.ny * self.nz

    def free_nodes(self):
        NX, NY, NZ = self.nx + 1, self.ny + 1, self.nz + 1
        if self.clamp_axis == 0:
            return NX * NY * NZ - NY * NZ
        return NX * NY * NZ - NX * NY


def _rng(tag: int) -> np.random.Generator:
    return np.random.default_rng([SEED, tag])


def cube16(n: int = 16) -> Problem:
    """Unit cube, n^3 elements, E = 1, nu = 0.3, z = 0 clamped, body load
    (0, 0, -1)."""
    h = 1.0 / n
    return Problem("cube%d" % n, n, n, n, h, h, h, 0.3, np.ones(n ** 3), 2, "body")


def beam(nx: int = 128, ny: int = 32, nz: int = 32) -> Problem:
    """Cantilever nx x ny x nz with unit elements, x = 0 clamped, tip shear of
    resultant -1 in z spread over the x = nx face, lognormal E (mu 0, sigma 1)
    per element, nu = 0.3."""
    E = np.exp(_rng(2).normal(0.0, 1.0, size=nx * ny * nz))
    return Problem("beam%dx%dx%d" % (nx, ny, nz), nx, ny, nz, 1.0, 1.0, 1.0, 0.3, E, 0,
                   "end_shear")


def slab(nx: int = 256, ny: int = 256, nz: int = 4) -> Problem:
    """Layered slab with element aspect 1:1:0.05, E = 1 and 1e4 in alternating
    element layers (bottom layer E = 1), nu = 0.45, z = 0 clamped, pressure
    U(0, 1) per top-face element pushing in -z."""
    layer = np.where(np.arange(nz) % 2 == 0, 1.0, 1e4)
    E = np.repeat(layer, nx * ny)
    p = _rng(3).uniform(0.0, 1.0, size=nx * ny)
    return Problem("slab%dx%dx%d" % (nx, ny, nz), nx, ny, nz, 1.0, 1.0, 0.05, 0.45, E, 2,
                   "top_pressure", pressure=p)


def cube_batched(n: int = 96, k: int = 64) -> Problem:
    """n^3 unit cube, E = 1, nu = 0.3, z = 0 clamped; k load cases of i.i.d.
    N(0, 1) forces (all three components) on every top-face node."""
    h = 1.0 / n
    nodal = _rng(4).normal(0.0, 1.0, size=(k, (n + 1) * (n + 1), 3))
    return Problem("cube%d_k%d" % (n, k), n, n, n, h, h, h, 0.3, np.ones(n ** 3), 2,
                   "top_nodal", nodal=nodal, nrhs=k)


def cube_simp(n: int = 128) -> Problem:
    """n^3 unit cube with SIMP densities rho_e ~ U(0.1, 1), E_e = rho_e^3,
    nu = 0.3, z = 0 clamped, body load (0, 0, -1); compliance f^T u."""
    h = 1.0 / n
    rho = _rng(5).uniform(0.1, 1.0, size=n ** 3)
    return Problem("simp%d" % n, n, n, n, h, h, h, 0.3, rho * rho * rho, 2, "body", rho=rho)


def beam6502k(nx: int = 512, ny: int = 64, nz: int = 64) -> Problem:
    """The paper's beam6502k (App. A.6), synthetic: a 8 x 1 x 1 cantilever of
    nx x ny x nz cubic elements (512 x 64 x 64: 2,097,152 elements,
    2,167,425 nodes), x = 0 face clamped, two materials along the length
    (first half E = 1e4, nu = 0.2; second half E = 1e7, nu = 0.4), and the
    paper's right-hand side of all ones (Sec. 4).  K_e = E_e Ke0(nu_e): each
    side assembles one matrix per Poisson ratio with the other material's
    moduli set to 0 and adds them."""
    h = 8.0 / nx
    ex = np.tile(np.arange(nx), ny * nz)
    first = ex < nx // 2
    E = np.where(first, 1e4, 1e7)
    nu_e = np.where(first, 0.2, 0.4)
    return Problem("beam6502k_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, h, h, h, 0.2, E, 0, "ones", nu_elem=nu_e)


CONFIGS = {
    "c1": cube16,
    "c2": beam,
    "c3": slab,
    "c4": cube_batched,
    "c5": cube_simp,
}


def fd_elements(p: Problem, count: int = 32) -> np.ndarray:
    """Seeded element ids for the finite-difference gradient check."""
    return np.sort(_rng(6).choice(p.ne, size=count, replace=False))


def padding_seed() -> int:
    """Seed of the counter-based generator that pads the near-null space and
    starts the Lanczos iterations."""
    return SEED
