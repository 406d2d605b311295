"""Seeded synthetic problem generators.

This module only builds inputs: the mesh description, the bed z sampled at
cell centres, the initial state, the boundary data and the solver parameters.
It holds none of the method's arithmetic, so both the CUDA library's tests and
the CPU oracle draw their inputs from here.

Conventions shared by both sides (interface only):
  * cell index i = ix + nx*iy, x fastest; cell centres x0 + (ix+1/2) dx;
  * states are SoA arrays of shape (ncomp, n): 1D (h, hu), 2D (h, hu, hv);
  * boundary sides are ordered W, E, S, N; a boundary's ``q`` is the discharge
    along the +axis direction (hu on W/E, hv on S/N), so an inflow at the west
    end has q > 0.

Workloads follow the paper's examples (Section 3) and the configurations the
benchmarks use: a seeded 1D bump (Example 3.2's bed), a 2D lake at rest with
dry islands, a 2D channel with Gaussian bumps and partial dry areas.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np

# boundary kinds (Remark 2.3)
BC_WALL_REFLECT = 0
BC_WALL_SLIP = 1
BC_INFLOW_DISCHARGE = 2
BC_OUTFLOW_DEPTH = 3
BC_SUPER_INFLOW = 4
BC_SUPER_OUTFLOW = 5
BC_AUTO_FROUDE = 6      # Remark 2.3 switch by the local Froude number

# numerical fluxes (Remark 2.2)
FLUX_HLL = 0
FLUX_HLLC = 1
FLUX_LLF = 2
FLUX_ROE = 3       # Roe with Harten's entropy fix (Remark 2.2)

INIT_CASCADE = 0   # Algorithm 1, Step 1
INIT_NONE = 1      # warm start from the given state

PREC_FP64 = 0
PREC_MIXED = 1     # FP32 multigrid inner solve, FP64 residual / update / norms
PREC_MIXED_STEP1 = 2   # PREC_MIXED, and Step 1's coarse-level BLU-SGS in FP32

SMOOTH_LEX = 0     # block SGS in lexicographic order (Section 2.3)
SMOOTH_COLOUR = 1  # variant: two colours, (ix + iy) even then odd

G = 9.81


@dataclass
class BC:
    kind: int = BC_WALL_REFLECT
    h: float = 0.0
    q: float = 0.0
    ut: float = 0.0


@dataclass
class Params:
    """Solver parameters; defaults are the paper's (Section 3 preamble)."""
    flux: int = FLUX_HLL
    llf_wetdry: int = 0
    alpha: float = 3.0
    fd_eps: float = 1e-8
    tau: float = 1.0
    h_eps: float = 1e-6
    eps_r: float = 0.03
    eps_p: float = 0.2
    tol: float = 1e-10
    n_levels: int = 3
    n_mg: int = 2
    nu1: int = 1
    nu2: int = 1
    gamma: int = 1
    coarse_sweeps: int = 8
    max_newton: int = 200
    max_blusgs: int = 1000
    init_mode: int = INIT_CASCADE
    precision: int = PREC_FP64
    eps_f: float = 0.4          # Harten's entropy-fix width (Roe flux)
    smoother: int = SMOOTH_LEX  # block SGS order (Section 2.3: lexicographic)

    def replace(self, **kw) -> "Params":
        return dataclasses.replace(self, **kw)


@dataclass
class Problem:
    name: str
    dim: int
    nx: int
    ny: int
    x0: float
    x1: float
    y0: float
    y1: float
    z: np.ndarray            # (n,) bed at cell centres
    U0: np.ndarray           # (ncomp, n) initial state
    bc: list                 # 4 BCs: W, E, S, N
    params: Params
    g: float = G
    meta: dict = field(default_factory=dict)
    # structured curvilinear quadrilateral mesh (2D only): vertex (a, b),
    # 0 <= a <= nx, 0 <= b <= ny, at (mesh_x[b, a], mesh_y[b, a]); None: the
    # uniform Cartesian mesh of [x0, x1] x [y0, y1]
    mesh_x: np.ndarray | None = None
    mesh_y: np.ndarray | None = None

    @property
    def ncomp(self) -> int:
        return 3 if self.dim == 2 else 2

    @property
    def n(self) -> int:
        return self.nx * (self.ny if self.dim == 2 else 1)

    def centres(self):
        if self.mesh_x is not None:           # mean of the four corners
            X = 0.25 * (self.mesh_x[:-1, :-1] + self.mesh_x[:-1, 1:] + self.mesh_x[1:, :-1] + self.mesh_x[1:, 1:])
            Y = 0.25 * (self.mesh_y[:-1, :-1] + self.mesh_y[:-1, 1:] + self.mesh_y[1:, :-1] + self.mesh_y[1:, 1:])
            return X.ravel(), Y.ravel()
        dx = (self.x1 - self.x0) / self.nx
        xc = self.x0 + (np.arange(self.nx) + 0.5) * dx
        if self.dim == 1:
            return xc
        dy = (self.y1 - self.y0) / self.ny
        yc = self.y0 + (np.arange(self.ny) + 0.5) * dy
        X, Y = np.meshgrid(xc, yc)            # (ny, nx): row iy, column ix
        return X.ravel(), Y.ravel()

    def with_params(self, **kw) -> "Problem":
        return dataclasses.replace(self, params=self.params.replace(**kw))


def _walls():
    return [BC(BC_WALL_REFLECT) for _ in range(4)]


# --------------------------------------------------------------------------- 1D

def bump_bed(x, a=0.2):
    """Bed of Example 3.2 (eq. bottom1) scaled to height a: a*max(0, 1-((x-10)/2)^2)."""
    return a * np.maximum(0.0, 1.0 - ((x - 10.0) / 2.0) ** 2)


def subcritical_bump_1d(seed: int = 101, n: int = 200, n_levels: int = 3) -> Problem:
    """1D subcritical flow over a seeded bump on [0, 25]: a ~ U[0.1, 0.2],
    inflow discharge q ~ U[4.0, 4.5] at x = 0, depth 2 at x = 25, initial
    h + z = 2 and u = 0; HLL flux, V-cycle, N_L levels."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.1, 0.2)
    q = rng.uniform(4.0, 4.5)
    p = Problem("bump1d", 1, n, 1, 0.0, 25.0, 0.0, 1.0, None, None, _walls(),
                Params(flux=FLUX_HLL, n_levels=n_levels, n_mg=2), meta={"a": a, "q": q, "seed": seed})
    x = p.centres()
    p.z = bump_bed(x, a)
    p.U0 = np.stack([2.0 - p.z, np.zeros(n)])
    p.bc[0] = BC(BC_INFLOW_DISCHARGE, q=q)
    p.bc[1] = BC(BC_OUTFLOW_DEPTH, h=2.0)
    return p


def smooth_subcritical_1d(n: int, flux: int = FLUX_HLL, n_levels: int = 3) -> Problem:
    """Example 3.1: z = 0.2 exp(-(x+1)^2/2) + 0.3 exp(-(x-1.5)^2) on [-10, 10],
    discharge hu = 1 at x = -10, depth h = 1 at x = 10."""
    p = Problem("ex31", 1, n, 1, -10.0, 10.0, 0.0, 1.0, None, None, _walls(),
                Params(flux=flux, n_levels=n_levels, n_mg=2))
    x = p.centres()
    p.z = 0.2 * np.exp(-(x + 1.0) ** 2 / 2.0) + 0.3 * np.exp(-(x - 1.5) ** 2)
    p.U0 = np.stack([1.0 - p.z, np.zeros(n)])
    p.bc[0] = BC(BC_INFLOW_DISCHARGE, q=1.0)
    p.bc[1] = BC(BC_OUTFLOW_DEPTH, h=1.0)
    return p


def transcritical_1d(n: int, case: int = 1, flux: int = FLUX_HLL, n_levels: int = 3) -> Problem:
    """Example 3.2 on [0, 25] with eq. bottom1: (I) q = 1.53, h_out = 0.66;
    (II) q = 0.18, h_out = 0.33."""
    q, hout = (1.53, 0.66) if case == 1 else (0.18, 0.33)
    p = Problem("ex32_%d" % case, 1, n, 1, 0.0, 25.0, 0.0, 1.0, None, None, _walls(),
                Params(flux=flux, n_levels=n_levels, n_mg=2))
    x = p.centres()
    p.z = bump_bed(x, 0.2)
    p.U0 = np.stack([np.maximum(hout - p.z, 0.0), np.zeros(n)])
    p.bc[0] = BC(BC_INFLOW_DISCHARGE, q=q)
    p.bc[1] = BC(BC_OUTFLOW_DEPTH, h=hout)
    return p


def wetdry_lake_1d(n: int, n_levels: int = 3, gamma: int = 1) -> Problem:
    """Example 3.3: bed of eq. bottom1 on [0, 20], initial h = 0.22 - z, u = 0,
    depth 0.1 imposed at both ends; LLF flux.  The steady state is
    h = max(0.1 - z, 0), u = 0."""
    p = Problem("ex33", 1, n, 1, 0.0, 20.0, 0.0, 1.0, None, None, _walls(),
                Params(flux=FLUX_LLF, llf_wetdry=1, n_levels=n_levels, n_mg=2, gamma=gamma))
    x = p.centres()
    p.z = bump_bed(x, 0.2)
    p.U0 = np.stack([0.22 - p.z, np.zeros(n)])
    p.bc[0] = BC(BC_OUTFLOW_DEPTH, h=0.1)
    p.bc[1] = BC(BC_OUTFLOW_DEPTH, h=0.1)
    return p


# --------------------------------------------------------------------------- 2D

def gaussian_bumps(X, Y, amp, width, cx, cy):
    """Sum of A exp(-((x-cx)^2 + (y-cy)^2) / (2 w^2)), w the standard deviation."""
    z = np.zeros_like(X)
    for A, w, x0, y0 in zip(amp, width, cx, cy):
        z += A * np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / (2.0 * w * w))
    return z


def lake_at_rest_2d(seed: int = 201, n: int = 256, flux: int = FLUX_LLF, n_levels: int = 3) -> Problem:
    """2D lake at rest with dry islands on [0,1]^2: 8 seeded Gaussian bumps
    (amplitude U[0.1, 0.6], width U[0.03, 0.15], centres U[0,1]^2), free
    surface 0.5, h = max(0, 0.5 - z), u = v = 0, reflective walls."""
    rng = np.random.default_rng(seed)
    amp = rng.uniform(0.1, 0.6, 8)
    wid = rng.uniform(0.03, 0.15, 8)
    cx = rng.uniform(0.0, 1.0, 8)
    cy = rng.uniform(0.0, 1.0, 8)
    p = Problem("lake2d", 2, n, n, 0.0, 1.0, 0.0, 1.0, None, None, _walls(),
                Params(flux=flux, llf_wetdry=1 if flux == FLUX_LLF else 0, n_levels=n_levels, n_mg=3,
                       init_mode=INIT_NONE), meta={"seed": seed})
    X, Y = p.centres()
    p.z = gaussian_bumps(X, Y, amp, wid, cx, cy)
    h = np.maximum(0.0, 0.5 - p.z)
    p.U0 = np.stack([h, np.zeros_like(h), np.zeros_like(h)])
    return p


def channel_2d(seed: int = 301, nx: int = 1024, ny: int = 1024, n_bumps: int = 16,
               q_range=(0.5, 1.5), n_levels: int = 3, precision: int = PREC_FP64,
               redraw: bool = True, dry_frac: float = 0.005) -> Problem:
    """2D steady channel flow with partial dry areas on [0,4]x[0,1]:
    n_bumps Gaussian bumps (amplitude U[0.05, 0.4], width U[0.03, 0.15],
    centre x U[0.4, 3.6], y U[0, 1]), inflow discharge hu ~ U[q_range] at
    x = 0, outflow depth 0.6 at x = 4, reflective walls at y = 0, 1; initial
    h = max(0, 0.6 - z), u = 0; LLF flux with the wet/dry speed increase.

    With ``redraw`` the bumps are redrawn with seed + 1000 k (k = 1, 2, ...)
    until at least ``dry_frac`` of the initial cells are dry on the fine grid
    and none of them lies in the first or last two columns; k is recorded in
    ``meta``.  The dry test is done on a 256-wide proxy grid so that the
    draw does not depend on the resolution."""
    def draw(s):
        rng = np.random.default_rng(s)
        amp = rng.uniform(0.05, 0.4, n_bumps)
        wid = rng.uniform(0.03, 0.15, n_bumps)
        cx = rng.uniform(0.4, 3.6, n_bumps)
        cy = rng.uniform(0.0, 1.0, n_bumps)
        q = rng.uniform(*q_range)
        return amp, wid, cx, cy, q

    def dry_ok(bumps):
        amp, wid, cx, cy, _ = bumps
        px, py = 256, 64
        xs = (np.arange(px) + 0.5) * (4.0 / px)
        ys = (np.arange(py) + 0.5) * (1.0 / py)
        X, Y = np.meshgrid(xs, ys)
        z = gaussian_bumps(X, Y, amp, wid, cx, cy)
        dry = z >= 0.6
        return dry.mean() >= dry_frac and not dry[:, :2].any() and not dry[:, -2:].any()

    k = 0
    bumps = draw(seed)
    while redraw and not dry_ok(bumps):
        k += 1
        bumps = draw(seed + 1000 * k)
        if k > 100000:
            raise RuntimeError("no dry draw found")
    amp, wid, cx, cy, q = bumps
    p = Problem("channel2d", 2, nx, ny, 0.0, 4.0, 0.0, 1.0, None, None, _walls(),
                Params(flux=FLUX_LLF, llf_wetdry=1, n_levels=n_levels, n_mg=3, precision=precision),
                meta={"seed": seed, "redraw_k": k, "q_in": q,
                      "bumps": (amp, wid, cx, cy)})
    X, Y = p.centres()
    p.z = gaussian_bumps(X, Y, amp, wid, cx, cy)
    h = np.maximum(0.0, 0.6 - p.z)
    p.U0 = np.stack([h, np.zeros_like(h), np.zeros_like(h)])
    p.bc[0] = BC(BC_INFLOW_DISCHARGE, q=q)
    p.bc[1] = BC(BC_OUTFLOW_DEPTH, h=0.6)
    return p


def supercritical_channel_2d(nx: int, ny: int, n_levels: int = 2, flux: int = FLUX_HLLC, froude: float = 2.5,
                             h0: float = 0.6, seed: int = 302) -> Problem:
    """A supercritical channel with every fixed open-boundary kind of
    Remark 2.3 that the partial-dry channel lacks: supercritical inflow at
    x = 0 (depth h0, discharge at the inflow Froude number, no tangential
    velocity), supercritical outflow at x = 4 and slip walls at y = 0, 1;
    six low Gaussian bumps (channel_2d's draw scaled by 0.3), initial state
    the inflow state everywhere."""
    p = channel_2d(seed=seed, nx=nx, ny=ny, n_bumps=6, n_levels=n_levels, redraw=False)
    p = p.with_params(flux=flux, llf_wetdry=0)
    q = h0 * froude * float(np.sqrt(p.g * h0))
    p.z = 0.3 * p.z
    p.U0 = np.stack([np.full(p.n, h0), np.full(p.n, q), np.zeros(p.n)])
    p.bc = [BC(BC_SUPER_INFLOW, h=h0, q=q, ut=0.0), BC(BC_SUPER_OUTFLOW), BC(BC_WALL_SLIP), BC(BC_WALL_SLIP)]
    p.meta = dict(p.meta, froude=froude)
    return p


def channel_bench(nx: int = 1024, ny: int = 1024, precision: int = PREC_MIXED, n_levels: int | None = None,
                  seed: int = 301) -> Problem:
    """The benchmark configuration of the partial-dry channel: channel_2d's
    input with W-cycles (gamma = 2), an exact solve of the coarsest level,
    N_mg = 3, eps_p = 2 and tol 1e-10.  The default level count coarsens to
    8 cells across (N_L = 7 at 1024^2)."""
    if n_levels is None:
        n_levels = max(0, min(nx, ny).bit_length() - 4)
    p = channel_2d(seed=seed, nx=nx, ny=ny, precision=precision)
    return p.with_params(gamma=2, eps_p=2.0, n_levels=n_levels, n_mg=3, coarse_sweeps=0, tol=1e-10,
                         max_newton=200)


def batch_channels(seed: int = 401, count: int = 64, sizes=(128, 256, 512, 1024), coarsest: int = 8,
                   precision: int = PREC_MIXED) -> list:
    """Batched workload: ``count`` independent channel problems.  A generator
    seeded with ``seed`` draws, per problem in order, the grid n x n with n
    uniform in ``sizes`` and the bump count uniform in 4..16; problem p then
    follows channel_2d with seed 1000 seed + p (bumps, inflow hu ~ U[0.3,
    1.5], the same dry redraw rule).  Levels: coarsest grid ``coarsest`` x
    ``coarsest`` (log2(n / coarsest) levels); W-cycles, eps_p = 2, exact
    coarsest solve, as for the single 1024 x 1024 workload."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(count):
        n = int(rng.choice(np.asarray(sizes)))
        nb = int(rng.integers(4, 17))
        nl = int(round(np.log2(n // coarsest)))
        pr = channel_2d(seed=1000 * seed + p, nx=n, ny=n, n_bumps=nb, q_range=(0.3, 1.5), n_levels=nl,
                        precision=precision)
        out.append(pr.with_params(gamma=2, eps_p=2.0, coarse_sweeps=0))
    return out


def transcritical_bump_2d(nx: int, ny: int, n_levels: int = 3) -> Problem:
    """Example 3.6: z = 0.2 - 0.05((x-10)^2 + y^2) inside radius 2 on
    [0,25]x[-5,5]; hu = 1.53 at x = 0, h = 0.52 at x = 25, reflective
    y-walls; HLLC flux, eps_p = 2."""
    p = Problem("ex36", 2, nx, ny, 0.0, 25.0, -5.0, 5.0, None, None, _walls(),
                Params(flux=FLUX_HLLC, n_levels=n_levels, n_mg=3, eps_p=2.0))
    X, Y = p.centres()
    r2 = (X - 10.0) ** 2 + Y ** 2
    p.z = np.where(r2 < 4.0, 0.2 - 0.05 * r2, 0.0)
    h = np.maximum(0.52 - p.z, 0.0)
    p.U0 = np.stack([h, np.zeros_like(h), np.zeros_like(h)])
    p.bc[0] = BC(BC_INFLOW_DISCHARGE, q=1.53)
    p.bc[1] = BC(BC_OUTFLOW_DEPTH, h=0.52)
    return p


def hill_wetdry_2d(nx: int, ny: int, n_levels: int = 3) -> Problem:
    """Example 3.7: hill z = 1.2 - 0.3((x-10)^2 + y^2) inside radius 2 on
    [0,25]x[-5,5]; hu = 0.1 at x = 0, h = 0.2 at x = 25, reflective y-walls,
    initial h = max(0.2 - z, 0) at rest; LLF flux."""
    p = Problem("ex37", 2, nx, ny, 0.0, 25.0, -5.0, 5.0, None, None, _walls(),
                Params(flux=FLUX_LLF, llf_wetdry=1, n_levels=n_levels, n_mg=3))
    X, Y = p.centres()
    r2 = (X - 10.0) ** 2 + Y ** 2
    p.z = np.where(r2 < 4.0, 1.2 - 0.3 * r2, 0.0)
    h = np.maximum(0.2 - p.z, 0.0)
    p.U0 = np.stack([h, np.zeros_like(h), np.zeros_like(h)])
    p.bc[0] = BC(BC_INFLOW_DISCHARGE, q=0.1)
    p.bc[1] = BC(BC_OUTFLOW_DEPTH, h=0.2)
    return p


# ------------------------------------------------------ curvilinear meshes

def cartesian_vertices(p: Problem):
    """Vertex arrays (ny+1, nx+1) of a 2D problem's uniform mesh."""
    xs = p.x0 + (p.x1 - p.x0) * (np.arange(p.nx + 1) / p.nx)
    ys = p.y0 + (p.y1 - p.y0) * (np.arange(p.ny + 1) / p.ny)
    X, Y = np.meshgrid(xs, ys)
    return X, Y


def with_mesh(p: Problem, X, Y) -> Problem:
    """The problem on the structured mesh with vertices (X, Y), each (ny+1, nx+1)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    assert p.dim == 2 and X.shape == Y.shape == (p.ny + 1, p.nx + 1)
    return dataclasses.replace(p, mesh_x=X, mesh_y=Y)


def _channel_mesh(nx: int, ny: int, length: float, half_width):
    """Vertices of a channel symmetric about y = 0: vertical mesh lines at
    x_a = length a/nx, each split into ny equal parts between -w(x_a) and
    w(x_a), w = half_width(x)."""
    xs = length * (np.arange(nx + 1) / nx)
    w = half_width(xs)
    frac = np.arange(ny + 1) / ny
    X = np.broadcast_to(xs, (ny + 1, nx + 1)).copy()
    Y = (2.0 * frac[:, None] - 1.0) * w[None, :]
    return X, Y


def constricted_channel(kind: str = "I", nx: int = 72, ny: int = 40, n_levels: int = 3,
                        flux: int = FLUX_HLLC) -> Problem:
    """Example 3.4: a flat channel of width 40 (y in [-20, 20]) and length 90,
    constricted symmetrically from x = 10 on at the angle 5 degrees to the end
    (channel I), or at 15 degrees up to x = 30 and straight after it (channel
    II).  Supercritical inflow h = 1, v = 0, Froude number 2.5 at x = 0,
    supercritical outflow at x = 90, slip walls; HLLC, V-cycle, N_L = 3,
    eps_p = 200.  The mesh's kinks (x = 10, 30) lie on vertices of every level
    when nx is a multiple of 9 * 2^N_L."""
    ang = np.deg2rad(5.0 if kind == "I" else 15.0)
    x_end = 90.0 if kind == "I" else 30.0

    def half_width(x):
        return 20.0 - (np.clip(x, 10.0, x_end) - 10.0) * np.tan(ang)

    X, Y = _channel_mesh(nx, ny, 90.0, half_width)
    u_in = 2.5 * np.sqrt(G * 1.0)
    n = nx * ny
    bc = [BC(BC_SUPER_INFLOW, h=1.0, q=u_in, ut=0.0), BC(BC_SUPER_OUTFLOW),
          BC(BC_WALL_SLIP), BC(BC_WALL_SLIP)]
    U0 = np.stack([np.ones(n), np.full(n, u_in), np.zeros(n)])
    p = Problem("ex34_" + kind, 2, nx, ny, 0.0, 90.0, -20.0, 20.0, np.zeros(n), U0, bc,
                Params(flux=flux, n_levels=n_levels, n_mg=3, eps_p=200.0, tol=1e-9),
                meta={"angle_deg": 5.0 if kind == "I" else 15.0, "froude_in": 2.5})
    return with_mesh(p, X, Y)


def hubbard_channel(froude: float, nx: int = 96, ny: int = 32, w_min: float = 0.9, h0: float = 1.0,
                    n_levels: int = 3, flux: int = FLUX_HLLC) -> Problem:
    """Example 3.5: a flat channel of length 3 and width
    W(x) = 1 - (1 - W_min) cos^2(pi (x - 1.5)) for |x - 1.5| <= 0.5, else 1,
    symmetric about y = 0.  Both open ends choose their condition by the local
    Froude number (Remark 2.3) with hu = h0 F_in sqrt(g h0), hv = 0 and
    h = h0 as the prescribed data; slip walls; initial state the inflow
    state; HLLC, V-cycle."""
    def half_width(x):
        s = x - 1.5
        return 0.5 * np.where(np.abs(s) <= 0.5, 1.0 - (1.0 - w_min) * np.cos(np.pi * s) ** 2, 1.0)

    X, Y = _channel_mesh(nx, ny, 3.0, half_width)
    q = h0 * froude * np.sqrt(G * h0)
    n = nx * ny
    bc = [BC(BC_AUTO_FROUDE, h=h0, q=q, ut=0.0), BC(BC_AUTO_FROUDE, h=h0, q=q, ut=0.0),
          BC(BC_WALL_SLIP), BC(BC_WALL_SLIP)]
    U0 = np.stack([np.full(n, h0), np.full(n, q), np.zeros(n)])
    p = Problem("ex35_F%g" % froude, 2, nx, ny, 0.0, 3.0, -0.5, 0.5, np.zeros(n), U0, bc,
                Params(flux=flux, n_levels=n_levels, n_mg=3),
                meta={"froude_in": froude, "w_min": w_min})
    return with_mesh(p, X, Y)


def random_state(p: Problem, seed: int, wet_frac: float = 1.0, u_scale: float = 0.3):
    """A seeded smooth-ish random state on p's grid for unit and parity tests:
    h = lake level + noise (dry where the bed is above it when wet_frac < 1),
    velocities of size u_scale."""
    rng = np.random.default_rng(seed)
    n = p.n
    eta = float(np.max(p.z)) * (1.0 if wet_frac >= 1.0 else 0.7) + 0.3
    h = np.maximum(eta - p.z + 0.05 * rng.standard_normal(n), 0.0)
    if wet_frac >= 1.0:
        h = np.maximum(h, 0.05)
    comps = [h]
    for _ in range(p.ncomp - 1):
        comps.append(h * u_scale * rng.standard_normal(n))
    U = np.stack(comps)
    U[:, h == 0.0] = 0.0
    return U


def adjoint_case(seed: int = 501, n: int = 512, n_gauges: int = 64, n_levels: int = 7):
    """Gradient workload: the partial-dry channel at n x n (FP64, W-cycles,
    exact coarsest solve), a loss over n_gauges distinct initially wet gauge
    cells L = sum (h + z - eta_obs)^2, where eta_obs comes from a forward
    solve on the bed with every bump amplitude scaled by (1 + 0.05 xi),
    xi ~ U[-1, 1].  Returns (problem, z_obs, gauge indices); eta_obs is
    computed by the caller's solver."""
    p = channel_2d(seed=seed, nx=n, ny=n, n_levels=n_levels)
    p = p.with_params(gamma=2, eps_p=2.0, coarse_sweeps=0)
    amp, wid, cx, cy = p.meta["bumps"]
    rng = np.random.default_rng(seed + 7)
    xi = rng.uniform(-1.0, 1.0, len(amp))
    X, Y = p.centres()
    z_obs = gaussian_bumps(X, Y, amp * (1.0 + 0.05 * xi), wid, cx, cy)
    wet = np.flatnonzero(p.U0[0] > 0.05)
    gauges = np.sort(rng.choice(wet, size=n_gauges, replace=False))
    return p, z_obs, gauges
