"""Seeded synthetic inputs for the generalized-Poisson pressure solve.

This module builds the *inputs* of one pressure solve: the densities
rho^n and rho^{n+1}, the squared sound speed c_s^2, the timestep dt and the
right-hand side f, on a cell-centred structured grid.  It holds none of the
solver's arithmetic (no coefficients c~ or kappa, no stencil): both the CUDA
path and the CPU oracle receive the arrays it returns.

Physical setting (paper Sec. 3.1-3.2): a hydrostatically stratified, ideal-gas
atmosphere spanning one pressure scale height, periodic horizontally and
walled vertically, gamma = 5/3.  The timestep follows the advective CFL rule
tau_fluid = CFL_adv * h / |u|_max of Sec. 2.6 with |u|_max = Ma * max c_s, so
the acoustic Courant number is CFL_adv / Ma.

Grids are stored row-major with x fastest: a 3D field has numpy shape
(nz, ny, nx) and a 2D field (nz, nx); the flat index is i + nx*(j + ny*k).
z is vertical (gravity along -z, z = 0 at the bottom), z in [0, 1] with
h = 1/nz, and cells are square (h_x = h_y = h_z).

Random numbers: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014), used as a
counter-based generator (output k of stream s is the SplitMix64 finaliser of
s + (k+1)*golden_gamma), turned into normals by Box-Muller.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GAMMA = 5.0 / 3.0          # adiabatic index of the ideal gas (Sec. 2, Table 1)
CFL_ADV = 0.5              # advective Courant number (Gresho test, Sec. 5)
BC_PERIODIC = 0
BC_NEUMANN = 1

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+count-1 of the SplitMix64 sequence seeded with `stream`."""
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(stream & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(stream: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(stream, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(stream: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller from two independent uniform streams."""
    u1 = 1.0 - uniform01(stream * 2 + 1, count)   # (0, 1]
    u2 = uniform01(stream * 2 + 2, count)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def _stream(seed: int, field: int) -> int:
    return (seed * 1_000_003 + field * 7919) & 0x7FFFFFFFFFFFFFFF


@dataclasses.dataclass
class Problem:
    """One generalized-Poisson solve: inputs plus the grid description."""
    n: tuple            # (nx, ny, nz); ny = 1 for 2D
    ndim: int
    h: tuple            # (hx, hy, hz)
    bc: tuple           # (bc_x, bc_y, bc_z), BC_PERIODIC or BC_NEUMANN
    rho_old: np.ndarray # rho^n, shape (nz, ny, nx) float64
    rho_new: np.ndarray # rho^{n+1}
    cs2: np.ndarray     # c_s^2 at time n
    dt: float
    f: np.ndarray       # right-hand side (per unit volume, units of c~ * P)
    rtol: float
    name: str = ""
    ma: float = 0.0

    @property
    def shape3(self):
        return (self.n[2], self.n[1], self.n[0])

    @property
    def size(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]


def smoothed_noise(shape3, bc, seed: int, sigma: float = 2.0, field: int = 1) -> np.ndarray:
    """White N(0,1) noise, Gaussian-smoothed (sigma in cells, radius 4 sigma;
    sigma = 0 leaves it white),
    wrapped on periodic axes and mirrored on walled axes, minus its mean and
    scaled to unit 2-norm."""
    from scipy import ndimage
    nz, ny, nx = shape3
    w = normal(_stream(seed, field), nz * ny * nx).reshape(shape3)
    if sigma <= 0.0:                       # white noise
        w -= w.mean()
        return w / np.linalg.norm(w)
    r = int(math.ceil(4 * sigma))
    t = np.arange(-r, r + 1, dtype=np.float64)
    g = np.exp(-0.5 * (t / sigma) ** 2)
    g /= g.sum()
    # numpy axis 2 = x, 1 = y, 0 = z
    for axis, b in ((2, bc[0]), (1, bc[1]), (0, bc[2])):
        if w.shape[axis] == 1:
            continue
        mode = "wrap" if b == BC_PERIODIC else "reflect"
        w = ndimage.convolve1d(w, g, axis=axis, mode=mode)
    w -= w.mean()
    nrm = np.linalg.norm(w)
    return w / nrm if nrm > 0 else w


def _z_centres(nz: int) -> np.ndarray:
    return (np.arange(nz, dtype=np.float64) + 0.5) / nz


def polytrope(nx: int, ny: int, nz: int, contrast: float | None = None, a: float | None = None):
    """Polytropic (n = 3/2) stratification over one unit of height:
    rho = (1 - a z)^1.5, P = (1 - a z)^2.5 (P_0 = rho_0 = 1 at the bottom),
    so the top/bottom density ratio is (1 - a)^1.5.  `contrast` = bottom/top
    density ratio fixes a = 1 - contrast^(-2/3)."""
    if a is None:
        a = 1.0 - contrast ** (-2.0 / 3.0)
    z = _z_centres(nz)
    base = 1.0 - a * z
    rho = np.broadcast_to((base ** 1.5)[:, None, None], (nz, ny, nx)).copy()
    P = np.broadcast_to((base ** 2.5)[:, None, None], (nz, ny, nx)).copy()
    return rho, P


def dt_from_mach(h: float, cs2: np.ndarray, ma: float) -> float:
    """Advective timestep CFL_adv * h / (Ma * max c_s)  (Sec. 2.6)."""
    return CFL_ADV * h / (ma * float(np.sqrt(cs2.max())))


def make_problem(nx: int, nz: int, ny: int = 1, *, ma: float, contrast: float | None = None,
                 a: float | None = None, noise: float = 0.0, rho_new_noise: float = 0.0,
                 seed: int = 1, rtol: float = 1e-8, bc=None, name: str = "") -> Problem:
    """Stratified-atmosphere problem: polytrope, optional relative density
    noise U(-1,1)*noise, c_s^2 = gamma P / rho, dt from Ma, smoothed-noise RHS."""
    ndim = 2 if ny == 1 else 3
    if bc is None:
        bc = (BC_PERIODIC, BC_PERIODIC, BC_NEUMANN)
    h = 1.0 / nz
    rho, P = polytrope(nx, ny, nz, contrast=contrast, a=a)
    if noise:
        xi = 2.0 * uniform01(_stream(seed, 2), rho.size).reshape(rho.shape) - 1.0
        rho = rho * (1.0 + noise * xi)
    cs2 = GAMMA * P / rho
    rho_new = rho.copy()
    if rho_new_noise:
        xi = 2.0 * uniform01(_stream(seed, 3), rho.size).reshape(rho.shape) - 1.0
        rho_new = rho * (1.0 + rho_new_noise * xi)
    dt = dt_from_mach(h, cs2, ma)
    f = smoothed_noise(rho.shape, bc, seed)
    return Problem(n=(nx, ny, nz), ndim=ndim, h=(h, h, h), bc=tuple(bc), rho_old=rho,
                   rho_new=rho_new, cs2=cs2, dt=dt, f=f, rtol=rtol, name=name, ma=ma)


# --- the workloads -----------------------------------------------------------

def config_plain_2d(n: int = 64, seed: int = 1) -> Problem:
    """2D n x n, x periodic / z walls, rho = (1 - 0.9 z)^1.5, Ma = 0.1, rtol 1e-10."""
    return make_problem(n, n, ma=0.1, a=0.9, seed=seed, rtol=1e-10,
                        name=f"plain2d-{n}x{n}-Ma0.1")


def config_convection_3d(n: int = 256, seed: int = 1) -> Problem:
    """3D n^3, x,y periodic / z walls, 20x density contrast + 1% noise, Ma = 0.01, rtol 1e-8."""
    return make_problem(n, n, n, ma=0.01, contrast=20.0, noise=0.01, seed=seed, rtol=1e-8,
                        name=f"convection3d-{n}^3-Ma0.01")


def batch_specs(count: int = 64, seed: int = 42, sides=(128, 256, 512, 1024), scale: int = 1):
    """Parameters of the uneven batch: (nx, nz) drawn independently from `sides`
    (divided by `scale` for downsized tests), Ma log-uniform in [1e-3, 1e-1],
    bottom/top density contrast uniform in [5, 30]."""
    u = uniform01(_stream(seed, 11), 4 * count).reshape(count, 4)
    specs = []
    for b in range(count):
        nx = sides[min(int(u[b, 0] * len(sides)), len(sides) - 1)] // scale
        nz = sides[min(int(u[b, 1] * len(sides)), len(sides) - 1)] // scale
        ma = 10.0 ** (-3.0 + 2.0 * u[b, 2])
        contrast = 5.0 + 25.0 * u[b, 3]
        specs.append(dict(nx=nx, nz=nz, ma=ma, contrast=contrast, seed=seed * 1000 + b))
    return specs


def config_batch(count: int = 64, seed: int = 42, scale: int = 1):
    return [make_problem(s["nx"], s["nz"], ma=s["ma"], contrast=s["contrast"], seed=s["seed"],
                         rtol=1e-8, name=f"batch-{b}-{s['nx']}x{s['nz']}")
            for b, s in enumerate(batch_specs(count, seed, scale=scale))]


TRAIN_SIGMAS = (0.0, 0.5, 1.0, 2.0, 4.0)


def config_training_2d(index: int, n: int = 256) -> Problem:
    """Member `index` of the learned-part family: n^2, contrast U[5,30],
    Ma log-uniform [1e-3, 1e-1], 1% density noise; the rhs smoothing width
    is drawn from TRAIN_SIGMAS (0 = white noise), because the network also
    preconditions inner residuals, which are rougher than the workloads'
    sigma = 2 right-hand sides."""
    u = uniform01(_stream(index, 13), 3)
    ma = 10.0 ** (-3.0 + 2.0 * u[0])
    contrast = 5.0 + 25.0 * u[1]
    sigma = TRAIN_SIGMAS[min(int(u[2] * len(TRAIN_SIGMAS)), len(TRAIN_SIGMAS) - 1)]
    p = make_problem(n, n, ma=ma, contrast=contrast, noise=0.01, seed=index, rtol=1e-8,
                     name=f"train2d-{index}-sigma{sigma}")
    p.f = smoothed_noise(p.shape3, p.bc, index, sigma=sigma).reshape(p.f.shape)
    return p


def semiconvection_profile(nz: int, a: float = 1.2, r_rho: float = 1.1, c_top: float = 0.2, g: float = 1.0,
                           R: float = 1.0, substeps: int = 64):
    """Two-component stratification over z in [0, 1] (Sec. 3.1): ideal gas
    P = R rho T / mu (Eq. idealEOS) with mu = 1/(c/4 + (1-c)/1), a linear
    temperature profile whose gradient is a times the adiabatic one of the
    top layer (b(x) = a, Eq. bfac; c_P = 2.5 R / mu), and a stabilising
    helium gradient with d ln mu / d ln P = R_rho (nabla - nabla_ad),
    nabla_ad = 1 - 1/gamma.  Hydrostatic equilibrium d ln P/dz = -g mu/(R T)
    is integrated downward from the top (P = 1, c = c_top) by classical RK4
    with `substeps` steps per cell.  Returns cell-centre (T, mu, P)."""
    mu_of = lambda c: 1.0 / (c / 4.0 + (1.0 - c))
    mu_top = mu_of(c_top)
    T_top = 1.0
    dTdz = -a * g * mu_top / (2.5 * R)          # T rises downward
    nabla_ad = 1.0 - 1.0 / GAMMA

    def rhs(z, y):
        lnP, lnmu = y
        T = T_top + dTdz * (z - 1.0)
        mu = math.exp(lnmu)
        dlnP = -g * mu / (R * T)
        nabla = (dTdz / T) / dlnP
        return np.array([dlnP, r_rho * (nabla - nabla_ad) * dlnP])

    h = 1.0 / nz
    zc = (np.arange(nz) + 0.5) * h
    out = np.zeros((nz, 2))
    y = np.array([0.0, math.log(mu_top)])
    z = 1.0
    k = nz - 1
    targets = list(zc[::-1])
    dz = -h / substeps
    # integrate from z = 1 down to each cell centre in turn
    for zt in targets:
        while z - zt > 1e-15:
            step = max(dz, zt - z)
            k1 = rhs(z, y)
            k2 = rhs(z + step / 2, y + step / 2 * k1)
            k3 = rhs(z + step / 2, y + step / 2 * k2)
            k4 = rhs(z + step, y + step * k3)
            y = y + step / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
            z += step
        out[k] = y
        k -= 1
    T = T_top + dTdz * (zc - 1.0)
    return T, np.exp(out[:, 1]), np.exp(out[:, 0])


def config_semiconvection_3d(n: int = 512, seed: int = 7, perturb: float = 0.01, ma: float = 0.001) -> Problem:
    """3D n^3 two-component semiconvection (Sec. 3.1, 3.3): the profile of
    semiconvection_profile, seeded relative perturbations U(-1,1)*perturb of
    T and of the helium fraction, rho = P mu / (R T), c_s^2 = gamma P / rho,
    dt at Ma = 0.001, x,y periodic, z walls, rtol 1e-8."""
    T0, mu0, P0 = semiconvection_profile(n)
    shape = (n, n, n)
    xiT = 2.0 * uniform01(_stream(seed, 21), n ** 3).reshape(shape) - 1.0
    xic = 2.0 * uniform01(_stream(seed, 22), n ** 3).reshape(shape) - 1.0
    T = T0[:, None, None] * (1.0 + perturb * xiT)
    c0 = (1.0 - 1.0 / mu0) / 0.75                  # helium fraction of the profile
    c = np.clip(c0[:, None, None] * (1.0 + perturb * xic), 0.0, 1.0)
    mu = 1.0 / (c / 4.0 + (1.0 - c))
    P = np.broadcast_to(P0[:, None, None], shape)
    rho = P * mu / T
    cs2 = GAMMA * P / rho
    del xiT, xic, T, c, mu
    h = 1.0 / n
    bc = (BC_PERIODIC, BC_PERIODIC, BC_NEUMANN)
    dt = dt_from_mach(h, cs2, ma)
    f = smoothed_noise(shape, bc, seed)
    return Problem(n=(n, n, n), ndim=3, h=(h, h, h), bc=bc, rho_old=rho, rho_new=rho.copy(), cs2=cs2, dt=dt,
                   f=f, rtol=1e-8, name=f"semiconvection3d-{n}^3-Ma{ma}", ma=ma)


def analytic_exp_problem(n: int, perturb: str | None = None, seed: int = 5, eps: float = 1e-2):
    """The stability test of Sec. 2.5.2 on [0,1]^2: -Lap(phi) + phi = 0 with
    phi = e^x, Neumann in x (d phi/dn = -1 at x = 0, e at x = 1), periodic in y.
    Returned as raw coefficient fields (ctilde, kappa per cell) plus the exact
    cell-centre solution; the wall flux data still has to be folded into f by
    the caller of the solver.  `perturb` in {None, 'f', 'kappa', 'c'} adds
    uniform noise of size eps to that field."""
    x = (np.arange(n) + 0.5) / n
    shape3 = (n, 1, n)            # numpy (y, 1, x): the paper's y plays our z slot
    ct = np.ones(shape3)
    kap = np.ones(shape3)
    f = np.zeros(shape3)
    xi = 2.0 * uniform01(_stream(seed, 17), n * n).reshape(shape3) - 1.0
    if perturb == "f":
        f = f + eps * xi
    elif perturb == "kappa":
        kap = kap * (1.0 + eps * xi)
    elif perturb == "c":
        ct = ct * (1.0 + eps * xi)
    exact = np.broadcast_to(np.exp(x)[None, None, :], shape3).copy()
    # axes: x Neumann (walls at x = 0, 1), second axis periodic
    bc = (BC_NEUMANN, BC_PERIODIC, BC_PERIODIC)
    return dict(n=(n, 1, n), h=(1.0 / n, 1.0, 1.0 / n), bc=bc, ctilde=ct, kappa=kap, f=f,
                exact=exact, g_low=-1.0, g_high=math.e)


def analytic_exp_problem_nodes(n: int, perturb: str | None = None, seed: int = 5, eps: float = 1e-2,
                               nper: int | None = None):
    """The Sec. 2.5.2 stability test on a grid of points for the finite-element
    operator: n points x_i = i / (n - 1) across [0,1] in x (the walls are
    points), `nper` points (default n - 1) around the periodic axis.  Same
    fields and noise as analytic_exp_problem, sampled at the points."""
    nper = n - 1 if nper is None else nper
    x = np.arange(n) / (n - 1)
    shape3 = (nper, 1, n)
    ct = np.ones(shape3)
    kap = np.ones(shape3)
    f = np.zeros(shape3)
    xi = 2.0 * uniform01(_stream(seed, 17), n * nper).reshape(shape3) - 1.0
    if perturb == "f":
        f = f + eps * xi
    elif perturb == "kappa":
        kap = kap * (1.0 + eps * xi)
    elif perturb == "c":
        ct = ct * (1.0 + eps * xi)
    exact = np.broadcast_to(np.exp(x)[None, None, :], shape3).copy()
    bc = (BC_NEUMANN, BC_PERIODIC, BC_PERIODIC)
    return dict(n=(n, 1, nper), h=(1.0 / (n - 1), 1.0, 1.0 / nper), bc=bc, ctilde=ct, kappa=kap, f=f,
                exact=exact, g_low=-1.0, g_high=math.e)


def gresho_vortex(n: int, ma: float, gamma: float = 5.0 / 3.0, cfl: float = 0.5) -> dict:
    """The Gresho vortex of Sec. 5.5.2 on a periodic n x n grid of cell
    centres over [0,1]^2 (the paper's y is this layout's z; arrays are
    (n, 1, n)): rho = 1, P0 = rho / (gamma Ma^2), the printed u_phi(r) and
    P(r), the velocity the counter-clockwise rotation u_phi (-sin t, cos t)
    with t = atan2(y - 1/2, x - 1/2), and total energy
    e = P / (gamma - 1) + rho |u|^2 / 2.  dt is the sound-speed-induced step
    cfl h / max(|u| + c_s) with c_s^2 = gamma P / rho."""
    h = 1.0 / n
    c = (np.arange(n) + 0.5) * h
    zz, xx = np.meshgrid(c, c, indexing="ij")
    dx, dz = xx - 0.5, zz - 0.5
    r = np.sqrt(dx * dx + dz * dz)
    t = np.arctan2(dz, dx)
    rho = np.ones((n, 1, n))
    p0 = 1.0 / (gamma * ma * ma)
    inner, ring = r <= 0.2, (r > 0.2) & (r <= 0.4)
    uphi = np.where(inner, 5.0 * r, np.where(ring, 2.0 - 5.0 * r, 0.0))
    rr = np.maximum(r, 1e-300)
    P = np.where(inner, p0 + 12.5 * r * r,
                 np.where(ring, p0 + 12.5 * r * r + 4.0 * (1.0 - 5.0 * r - math.log(0.2) + np.log(rr)),
                          p0 - 2.0 + 4.0 * math.log(2.0)))
    ux = (-np.sin(t) * uphi)[:, None, :]
    uz = (np.cos(t) * uphi)[:, None, :]
    P = P[:, None, :]
    mom = [rho * ux, np.zeros_like(rho), rho * uz]
    e = P / (gamma - 1.0) + 0.5 * rho * (ux * ux + uz * uz)
    cs = np.sqrt(gamma * P / rho)
    dt = cfl * h / float(np.max(np.sqrt(ux * ux + uz * uz) + cs))
    return dict(n=(n, 1, n), h=(h, 1.0, h), bc=(BC_PERIODIC, BC_PERIODIC, BC_PERIODIC), rho=rho, mom=mom, e=e,
                P=P, gamma=gamma, dt=dt, ma=ma, name=f"gresho-{n}^2-Ma{ma}")
