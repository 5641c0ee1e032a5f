"""Seeded synthetic workloads: problem descriptors shared by the oracle and the CUDA path.

This module only *describes* inputs (mesh sizes, material constants, boundary data, load
schedules, random draws).  It contains none of the solver's arithmetic: the oracle and the GPU
library each turn a :class:`Workload` into their own data structures.

Coordinates of the structured meshes are given in *doubled grid units*: a vertex (i, j) has
doubled coordinates (2i, 2j); a cell-centre node of a crossed mesh has (2i+1, 2j+1).  Boundary
pins and damage boxes are stated in these integer units so that both sides select exactly the
same nodes.

Problem set-ups follow the paper's test cases (Section 4): traction of a bar (Section 4.2), a
single-edge notched square (Mode I, a standard variant of the paper's smooth-propagation tests)
and the thermal shock slab (Section 4.3, eqs. energytshock and tempfielderfc).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Dict, List, Optional, Tuple

import numpy as np

EDGES = ("left", "right", "bottom", "top")
E_DEFAULT, GC_DEFAULT = 1.0, 1.0  # Young's modulus and toughness of every workload
COMPS = ("ux", "uy", "alpha")


@dataclass
class Workload:
    """One quasi-static fracture problem on a structured P1 triangulation.

    fixed[edge][comp] = g means the component is prescribed on that edge with value t*g for
    displacement components (t = load amplitude of the step) and value g for the damage.
    pins: (x2, y2, comp, g) single prescribed nodes in doubled grid units.
    alpha_boxes: (x2_lo, x2_hi, y2_lo, y2_hi, value): nodes inside get alpha = alpha_prev = value
    initially (a pre-existing crack when value = 1, Section 4 notch; a seed otherwise).
    loads: list of (t, dT): displacement amplitude and thermal shock amplitude per load step.
    """

    name: str
    kind: str  # "right" | "crossed"
    nx: int
    ny: int
    x0: float
    y0: float
    lx: float
    ly: float
    E: float = 1.0
    nu: float = 0.3
    Gc: float = 1.0
    ell: float = 0.05
    k_ell: float = 1e-6
    model: str = "AT1"  # "AT1" | "AT2"
    plane: str = "strain"  # "strain" | "stress"
    beta: float = 0.0  # thermal expansion coefficient
    pen: float = 1.0  # thermal penetration length 2*sqrt(kappa*t) (Section 4.3)
    fixed: Dict[str, Dict[str, float]] = field(default_factory=dict)
    pins: List[Tuple[int, int, str, float]] = field(default_factory=list)
    alpha_boxes: List[Tuple[int, int, int, int, float]] = field(default_factory=list)
    loads: List[Tuple[float, float]] = field(default_factory=list)
    omega: float = 1.0
    # Prescribed displacements that follow a moving Mode-I crack tip (Section 4.1): when set,
    # dict(KI=stress intensity factor, x_tip0=tip abscissa at t = 0, v=tip speed, y_line=crack
    # line ordinate); the prescribed value of component c on a fixed edge is then
    # g * u_bar_c(x - x_tip0 - v t, y - y_line) instead of t * g.
    mode_I: Optional[Dict[str, float]] = None

    @property
    def hx(self) -> float:
        return self.lx / self.nx

    @property
    def hy(self) -> float:
        return self.ly / self.ny

    def n_nodes(self) -> int:
        nv = (self.nx + 1) * (self.ny + 1)
        return nv + (self.nx * self.ny if self.kind == "crossed" else 0)

    def n_elements(self) -> int:
        return self.nx * self.ny * (4 if self.kind == "crossed" else 2)

    def with_loads(self, loads) -> "Workload":
        return replace(self, loads=list(loads))


# ---------------------------------------------------------------------------------------------
# Critical loads used to place the load schedules (closed forms of the model stated in Section 4,
# in plane strain: the homogeneous states have q = E/(1-nu^2) eps^2, so the AT1 onset
# q = 3 Gc/(8 ell) gives t_c and dT_c below).  These only position the inputs.
# ---------------------------------------------------------------------------------------------
def plane_strain_modulus(E: float, nu: float) -> float:
    return E / (1.0 - nu * nu)


def bar_critical_displacement(L: float, E: float, nu: float, Gc: float, ell: float,
                              plane: str = "strain") -> float:
    """t_c of the AT1 bar (Section 4.2), with E replaced by E/(1-nu^2) in plane strain."""
    Eeff = plane_strain_modulus(E, nu) if plane == "strain" else E
    return L * math.sqrt(3.0 * Gc / (8.0 * Eeff * ell))


def thermal_critical_jump(E: float, nu: float, Gc: float, ell: float, beta: float) -> float:
    """Damage-onset amplitude of the AT1 thermal shock in plane strain (Section 4.3 reading)."""
    return math.sqrt(3.0 * Gc * (1.0 - nu * nu) / (8.0 * E * ell)) / beta


# ---------------------------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------------------------
def bar(nx: int = 128, ny: int = 16, n_steps: int = 20, ell: float = 0.05, model: str = "AT1",
        nu: float = 0.3, lx: float = 1.0, ly: float = 0.1, seed_column: bool = False,
        load_factor: float = 1.5, k_ell: float = 1e-6) -> Workload:
    """Uniaxial traction of a bar (Section 4.2): x=0: u_x=0, alpha=0; x=L: u_x=t, alpha=0;
    u_y=0 at the left mid-height node; loads t_k = load_factor*t_c*k/n_steps."""
    if ny % 2:
        raise ValueError("ny must be even (mid-height pin)")
    tc = bar_critical_displacement(lx, 1.0, nu, 1.0, ell)
    loads = [(load_factor * tc * k / n_steps, 0.0) for k in range(1, n_steps + 1)]
    boxes = []
    if seed_column:  # symmetry-breaking seed on the vertex column one cell right of x = L/2
        # (x = L/2 itself is the centre of the mesh's 180-degree rotation symmetry)
        if nx % 2:
            raise ValueError("nx must be even for the seed column")
        boxes.append((nx + 2, nx + 2, 0, 2 * ny, 1e-3))
    return Workload(
        name=f"bar_{nx}x{ny}", kind="right", nx=nx, ny=ny, x0=0.0, y0=0.0, lx=lx, ly=ly,
        nu=nu, ell=ell, model=model, k_ell=k_ell,
        fixed={"left": {"ux": 0.0, "alpha": 0.0}, "right": {"ux": 1.0, "alpha": 0.0}},
        pins=[(0, ny, "uy", 0.0)], alpha_boxes=boxes, loads=loads, omega=1.0)


def notched_square(n: int = 512, n_steps: int = 50, t_max: float = 2.0, ell_over_h: float = 4.0,
                   model: str = "AT1", nu: float = 0.3, omega: float = 1.5,
                   k_ell: float = 1e-6) -> Workload:
    """Single-edge notched unit square in Mode I on an n x n crossed mesh: notch x <= 0.5,
    |y - 0.5| <= h (two elements wide); bottom clamped; top u_x = 0, u_y = t; sides free;
    t_k = k t_max / n_steps.  With t_max = 2 the crack starts near t = 1.2-1.3 (AT1, ell = 4h,
    E = Gc = 1) and crosses the ligament before the last step."""
    if n % 2:
        raise ValueError("n must be even")
    h = 1.0 / n
    loads = [(t_max * k / n_steps, 0.0) for k in range(1, n_steps + 1)]
    notch = (0, n, n - 2, n + 2, 1.0)  # doubled units: X2 <= n (x <= 0.5), |Y2 - n| <= 2
    return Workload(
        name=f"notched_{n}", kind="crossed", nx=n, ny=n, x0=0.0, y0=0.0, lx=1.0, ly=1.0,
        nu=nu, ell=ell_over_h * h, model=model, k_ell=k_ell,
        fixed={"bottom": {"ux": 0.0, "uy": 0.0}, "top": {"ux": 0.0, "uy": 1.0}},
        alpha_boxes=[notch], loads=loads, omega=omega)


def thermal_shock(nx: int = 1024, ny: int = 256, n_steps: int = 40, ell_over_h: float = 3.0,
                  max_ratio: float = 4.0, pen_over_ell: float = 10.0, model: str = "AT1",
                  nu: float = 0.3, omega: float = 1.6, k_ell: float = 1e-6) -> Workload:
    """Thermal shock slab [-0.5,0.5]x[0,0.25] (Section 4.3): top u = 0; sides u_x = 0; bottom
    free; no damage Dirichlet data; dT_k = k*max_ratio*dT_c/n_steps; right-triangle cells."""
    lx, ly = 1.0, ly_default(nx, ny)
    h = lx / nx
    ell = ell_over_h * h
    dtc = thermal_critical_jump(1.0, nu, 1.0, ell, 1.0)
    loads = [(0.0, max_ratio * dtc * k / n_steps) for k in range(1, n_steps + 1)]
    return Workload(
        name=f"thermal_{nx}x{ny}", kind="right", nx=nx, ny=ny, x0=-0.5, y0=0.0, lx=lx, ly=ly,
        nu=nu, ell=ell, model=model, beta=1.0, pen=pen_over_ell * ell, k_ell=k_ell,
        fixed={"top": {"ux": 0.0, "uy": 0.0}, "left": {"ux": 0.0}, "right": {"ux": 0.0}},
        loads=loads, omega=omega)


def surfing(nx: int = 200, ny: int = 100, ell: float = 0.05, n_steps: int = 30,
            t_max: float = 1.2, model: str = "AT1", kind: str = "crossed", nu: float = 0.3,
            omega: float = 1.6, k_ell: float = 1e-6, crack_length: float = 0.05,
            speed: float = 1.0, ki_ratio: float = 1.0) -> Workload:
    """Surfing (Section 4.1): slab [0, 2] x [-1/2, 1/2], plane stress, the asymptotic Mode-I
    displacement of eq. (surfingloading) prescribed on the whole boundary with its tip at
    x = crack_length + speed * t; K_I = ki_ratio * sqrt(Gc E); a pre-existing crack (alpha = 1)
    on the nodes with x <= crack_length and |y| <= h; loads t_k = k t_max / n_steps."""
    if ny % 2:
        raise ValueError("ny must be even (crack line y = 0 on the grid)")
    lx, ly = 2.0, 1.0
    hx = lx / nx
    loads = [(t_max * k / n_steps, 0.0) for k in range(1, n_steps + 1)]
    x2c = int(round(2 * crack_length / hx))
    crack = (0, x2c, ny - 2, ny + 2, 1.0)
    fix = {"ux": 1.0, "uy": 1.0}
    return Workload(
        name=f"surfing_{nx}x{ny}_ell{ell:g}", kind=kind, nx=nx, ny=ny, x0=0.0, y0=-0.5, lx=lx,
        ly=ly, nu=nu, ell=ell, model=model, k_ell=k_ell, plane="stress",
        fixed={e: dict(fix) for e in EDGES}, alpha_boxes=[crack], loads=loads, omega=omega,
        mode_I=dict(KI=ki_ratio * math.sqrt(GC_DEFAULT * E_DEFAULT), x_tip0=crack_length,
                    v=speed, y_line=0.0))


def ly_default(nx: int, ny: int) -> float:
    """Slab height keeping square cells (1 x 0.25 for 1024 x 256)."""
    return ny / nx


def batch_of_notched(n_instances: int = 256, lo: int = 64, hi: int = 256, seed: int = 0,
                     multiple: int = 16, n_steps: int = 50, t_max: float = 2.0) -> List[Workload]:
    """Batched notched squares: N log-uniform on [lo, hi] rounded to a multiple of 16, ell
    uniform in [2h, 8h], nu uniform in [0.2, 0.35]; one step each to t ~ U[0.5, 1.0]*t_max."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(n_instances):
        n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        n = max(multiple, int(round(n / multiple)) * multiple)
        ell_over_h = float(rng.uniform(2.0, 8.0))
        nu = float(rng.uniform(0.2, 0.35))
        t = float(rng.uniform(0.5, 1.0)) * t_max
        w = notched_square(n=n, n_steps=1, t_max=t, ell_over_h=ell_over_h, nu=nu, omega=1.6)
        w.name = f"batch{b}_notched_{n}"
        out.append(w)
    return out


@dataclass
class Job:
    """One serving request: a workload and its arrival time (seconds)."""

    job_id: int
    arrival: float
    workload: Workload


def serving_stream(n_jobs: int = 64, rate: float = 4.0, seed: int = 0, lo: int = 32,
                   hi: int = 1024, multiple: int = 16, min_steps: int = 10,
                   max_steps: int = 60) -> List[Job]:
    """Poisson arrivals of notched-square and bar jobs; N log-uniform on [lo, hi] (multiple of
    16); 10..60 load steps each."""
    rng = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    for k in range(n_jobs):
        t += float(rng.exponential(1.0 / rate))
        n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        n = max(multiple, int(round(n / multiple)) * multiple)
        steps = int(rng.integers(min_steps, max_steps + 1))
        if rng.uniform() < 0.5:
            w = notched_square(n=n, n_steps=steps, omega=1.6)
        else:
            nb = max(8 * multiple, n)
            nb = int(round(nb / (8 * multiple))) * 8 * multiple
            w = bar(nx=nb, ny=nb // 8, n_steps=steps)
        jobs.append(Job(job_id=k, arrival=t, workload=w))
    return jobs


def random_fields(w: Workload, seed: int, alpha_max: float = 1.0, u_scale: float = 1.0):
    """Seeded random nodal fields (u interleaved (n,2), alpha (n,)) for operator parity tests."""
    rng = np.random.default_rng(seed)
    n = w.n_nodes()
    u = rng.uniform(-u_scale, u_scale, size=(n, 2))
    alpha = rng.uniform(0.0, alpha_max, size=n)
    return u, alpha
