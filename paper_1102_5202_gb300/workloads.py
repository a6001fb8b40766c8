"""Seeded synthetic inputs: primitive states and metrics of the benchmark and test problems.

This module holds no step of the finite-volume method.  It only writes initial primitive
fields (rho, p, u~^i, B^i, psi) and the metric (alpha, beta^i, gamma_ij) at cell centres, so
that the CUDA library and the FP64 oracle can be fed identical inputs.  The conserved state
is computed from these on each side by its own code.

Layouts (float64, C-contiguous):
  prim   (9, nz, ny, nx)                     fields rho, p, u~x, u~y, u~z, Bx, By, Bz, psi
  metric (10, nz+2gz, ny+2gy, nx+2gx)        fields alpha, beta^x,y,z, g_xx,xy,xz,yy,yz,zz
where g? = 1 on an axis with more than one cell (one ghost layer of true metric values) and 0
otherwise.  u~^i = W v^i is the primitive velocity of the paper (§5.2 footnote), v^i the
Eulerian three-velocity; B^i = *F^{it} (§2.1).

Workloads (sizes, states and seeds are those of the benchmark configurations):
  * ``balsara1``   1-D magnetised shock tube, N=400 on [-0.5, 0.5], Gamma = 2, t = 0.4 (§5.1);
  * ``sod``        1-D unmagnetised relativistic shock tube, Gamma = 5/3 (§5.1);
  * ``blob3d``     3-D rotating polytropic-like blob in a capped isotropic Schwarzschild
                   metric (stand-in for the paper's rns neutron-star model of §4.1, which needs
                   the external rns code), seed 1102;
  * ``ensemble``   512 independent 1-D magnetised tubes of uneven size, seed 1103;
  * random pointwise states and metrics for recovery and flux tests.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

PRIM_FIELDS = ("rho", "p", "utx", "uty", "utz", "Bx", "By", "Bz", "psi")
CONS_FIELDS = ("D", "Tt", "Tx", "Ty", "Tz", "BBx", "BBy", "BBz", "Psi")
METRIC_FIELDS = ("alp", "betax", "betay", "betaz", "gxx", "gxy", "gxz", "gyy", "gyz", "gzz")
BC_OUTFLOW, BC_PERIODIC = 0, 1


@dataclasses.dataclass
class Problem:
    name: str
    n: Tuple[int, int, int]                 # (nx, ny, nz)
    dx: Tuple[float, float, float]
    x0: Tuple[float, float, float]          # coordinate of the lower domain face
    bc: Tuple[int, int, int]
    gamma: float
    prim: np.ndarray                        # (9, nz, ny, nx)
    metric: np.ndarray                      # (10, nz+2gz, ny+2gy, nx+2gx)
    t_end: float = 0.0
    cfl: float = 0.5
    cleaning: bool = False
    ch: float = 0.0
    kappa: float = 0.0
    rho_floor: float = 1e-12
    rho_atm: float = 0.0                    # atmosphere threshold on D / sqrt(gamma) (0: off)
    p_floor: float = 1e-14
    atm_K: float = 0.0
    steps: int = 0                          # fixed step count of the benchmark problems
    recon: int = 0                          # reconstruction: 0 MC, 1 PPM (§3.2)
    c2p: int = 0                            # GPU recovery scheme: 0 2D Newton, 1 1D Newton (§3.2)

    @property
    def ncell(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    def ghosts(self) -> Tuple[int, int, int]:
        return tuple(1 if k > 1 else 0 for k in self.n)

    def subbox(self, lo: Sequence[int], hi: Sequence[int], name: str = "") -> "Problem":
        """Cells lo <= (i, j, k) < hi as a problem of its own: primitives, the metric with its
        ghost layer, and every option; boundaries stay those of the parent."""
        g = self.ghosts()
        prim = np.ascontiguousarray(self.prim[:, lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]])
        met = np.ascontiguousarray(self.metric[:, lo[2]:hi[2] + 2 * g[2], lo[1]:hi[1] + 2 * g[1],
                                               lo[0]:hi[0] + 2 * g[0]])
        x0 = tuple(self.x0[d] + lo[d] * self.dx[d] for d in range(3))
        n = tuple(int(hi[d] - lo[d]) for d in range(3))
        return dataclasses.replace(self, name=name or f"{self.name}_sub", n=n, x0=x0, prim=prim,
                                   metric=met)


def metric_ghosts(n: Sequence[int]) -> Tuple[int, int, int]:
    return tuple(1 if k > 1 else 0 for k in n)


def centre_coords(n, dx, x0, with_ghost: bool):
    """Cell-centre coordinates per axis (with the metric's ghost layer when asked)."""
    out = []
    for d in range(3):
        g = (1 if n[d] > 1 else 0) if with_ghost else 0
        idx = np.arange(-g, n[d] + g, dtype=np.float64)
        out.append(x0[d] + (idx + 0.5) * dx[d])
    return out


def minkowski_metric(n: Sequence[int]) -> np.ndarray:
    gx, gy, gz = metric_ghosts(n)
    shape = (n[2] + 2 * gz, n[1] + 2 * gy, n[0] + 2 * gx)
    m = np.zeros((10,) + shape)
    m[0] = 1.0
    m[4] = m[7] = m[9] = 1.0
    return m


def _tube_prim(n: int, left: dict, right: dict, xs: np.ndarray, x_split: float) -> np.ndarray:
    """Piecewise-constant 1-D primitives from states given with Eulerian velocity v^i."""
    prim = np.zeros((9, n))
    for side, mask in ((left, xs < x_split), (right, xs >= x_split)):
        v = np.array([side.get("vx", 0.0), side.get("vy", 0.0), side.get("vz", 0.0)])
        W = 1.0 / math.sqrt(1.0 - float(v @ v))
        vals = [side["rho"], side["p"], W * v[0], W * v[1], W * v[2],
                side.get("Bx", 0.0), side.get("By", 0.0), side.get("Bz", 0.0), 0.0]
        for f in range(9):
            prim[f, mask] = vals[f]
    return prim


def shock_tube(n: int, left: dict, right: dict, gamma: float, t_end: float, axis: int = 0,
               lo: float = -0.5, hi: float = 0.5, name: str = "tube", cfl: float = 0.5) -> Problem:
    """1-D Riemann problem along ``axis`` (the other two axes have one cell), Minkowski."""
    dx = (hi - lo) / n
    xs = lo + (np.arange(n) + 0.5) * dx
    p1 = _tube_prim(n, left, right, xs, 0.5 * (lo + hi))
    if axis != 0:
        # rotate vector components so that the tube normal is ``axis``
        perm = {1: (1, 2, 0), 2: (2, 0, 1)}[axis]  # old component k becomes component perm[k]
        q = p1.copy()
        for k in range(3):
            q[2 + perm[k]] = p1[2 + k]
            q[5 + perm[k]] = p1[5 + k]
        p1 = q
    shape3 = [1, 1, 1]
    shape3[axis] = n
    nn = tuple(shape3)  # (nx, ny, nz)
    prim = p1.reshape((9, nn[2], nn[1], nn[0]))
    dxs = [1.0, 1.0, 1.0]
    dxs[axis] = dx
    x0 = [0.0, 0.0, 0.0]
    x0[axis] = lo
    return Problem(name=name, n=nn, dx=tuple(dxs), x0=tuple(x0), bc=(0, 0, 0), gamma=gamma,
                   prim=np.ascontiguousarray(prim), metric=minkowski_metric(nn), t_end=t_end,
                   cfl=cfl)


BALSARA1_LEFT = dict(rho=1.0, p=1.0, Bx=0.5, By=1.0, Bz=0.0)
BALSARA1_RIGHT = dict(rho=0.125, p=0.1, Bx=0.5, By=-1.0, Bz=0.0)
SOD_LEFT = dict(rho=1.0, p=1.0)
SOD_RIGHT = dict(rho=0.125, p=0.1)


def balsara1(n: int = 400, axis: int = 0, gamma: float = 2.0, t_end: float = 0.4) -> Problem:
    """Magnetised shock tube (first Balsara test, §5.1) with the benchmark's Gamma=2, t=0.4."""
    return shock_tube(n, BALSARA1_LEFT, BALSARA1_RIGHT, gamma, t_end, axis=axis, name="balsara1")


def sod(n: int = 400, axis: int = 0, gamma: float = 5.0 / 3.0, t_end: float = 0.4) -> Problem:
    """Relativistic Sod tube (§5.1: rho, P = 1, 1 | 0.125, 0.1, Gamma = 5/3)."""
    return shock_tube(n, SOD_LEFT, SOD_RIGHT, gamma, t_end, axis=axis, name="sod")


# ------------------------------------------------------------------ 3-D blob (rns stand-in)
BLOB_M = 1.4
BLOB_R = 8.0
BLOB_K = 100.0
BLOB_GAMMA = 2.0
BLOB_RHOC = 1.28e-3
BLOB_OMEGA = 0.02
BLOB_ATM = 1e-10


def capped_radius(r: np.ndarray) -> np.ndarray:
    """r for r >= 8; inside, 8 (3/8 + 3/4 s^2 - 1/8 s^4) with s = r/8 (C^2 at r = 8, >= 3)."""
    s = r / BLOB_R
    inner = BLOB_R * (3.0 / 8.0 + 0.75 * s * s - 0.125 * s ** 4)
    return np.where(r >= BLOB_R, r, inner)


def blob_metric_fields(x, y, z):
    """Isotropic Schwarzschild-exterior lapse and conformal factor with the capped radius."""
    r = np.sqrt(x * x + y * y + z * z)
    re = capped_radius(r)
    h = BLOB_M / (2.0 * re)
    alp = (1.0 - h) / (1.0 + h)
    psi4 = (1.0 + h) ** 4
    return alp, psi4


# Gauss per code unit of field strength (G = c = M_sun = 1, Heaviside-Lorentz, magnetic
# pressure b^2/2): b^2/2 = B_G^2 / (8 pi) / e_unit with e_unit = (M_sun / L^3) c^2 and
# L = G M_sun / c^2, so B_code = B_G / sqrt(4 pi e_unit).
GAUSS_PER_CODE_UNIT = 8.352e19
TOROIDAL_B_GAUSS = 2.6e15      # largest field strength of the toroidal model (§5.2)
TOROIDAL_VARPI0 = 3.0
TOROIDAL_H = 1.0


def toroidal_profile(X, Y, Z, varpi0: float = TOROIDAL_VARPI0, H: float = TOROIDAL_H):
    """Field strength profile (varpi/varpi0)^2 exp(-varpi^2/varpi0^2) exp(-z^2/(2 H^2)) of the
    toroidal model of §5.2.  The paper prints the last factor as exp(-z/2H), which is not even
    in z; it is read as exp(-z^2/(2 H^2)).  The profile peaks at varpi = varpi0, z = 0 with
    the value 1/e."""
    w2 = (X * X + Y * Y) / (varpi0 * varpi0)
    return w2 * np.exp(-w2) * np.exp(-Z * Z / (2.0 * H * H))


def blob3d(n: int = 192, seed: int = 1102, half_width: float = 20.0, kappa: float = 1.0,
           ch: float = 0.5, cleaning: bool = True, steps: int = 100, field: str = "poloidal") -> Problem:
    """3-D rotating blob in a fixed curved spacetime (G = c = M_sun = 1).

    rho = rho_c (max(1 - (r/8)^2, 0) + 1e-10)(1 + 0.01 xi), xi ~ U[-1, 1] per cell (seeded);
    p = K rho_unperturbed^Gamma; coordinate velocity Omega (-y, x, 0) inside r < 8.
    field = "poloidal": B from A_phi = A_b max(p - 0.04 p_max, 0) varpi^2, with A_b scaled so
    that the largest Eulerian magnetic pressure is 1e-3 of the largest gas pressure.
    field = "toroidal": the toroidal model of §5.2, Eulerian field B_n = B0 toroidal_profile e_phi
    (unit vector of the spatial metric), B0 = e * 2.6e15 G so that the largest field strength is
    2.6e15 G; B^z = 0 and sqrt(gamma) B^i is divergence-free (an axisymmetric toroidal field).
    """
    nn = (n, n, n)
    dx = 2.0 * half_width / n
    x0 = (-half_width,) * 3
    # metric with ghosts
    cx, cy, cz = centre_coords(nn, (dx,) * 3, x0, with_ghost=True)
    Z, Y, X = np.meshgrid(cz, cy, cx, indexing="ij")
    alp, psi4 = blob_metric_fields(X, Y, Z)
    met = np.zeros((10,) + X.shape)
    met[0] = alp
    met[4] = met[7] = met[9] = psi4
    # interior centres
    cx, cy, cz = centre_coords(nn, (dx,) * 3, x0, with_ghost=False)
    Z, Y, X = np.meshgrid(cz, cy, cx, indexing="ij")
    alp_c, psi4_c = blob_metric_fields(X, Y, Z)
    r = np.sqrt(X * X + Y * Y + Z * Z)
    prof = np.maximum(1.0 - (r / BLOB_R) ** 2, 0.0) + BLOB_ATM
    rho0 = BLOB_RHOC * prof
    rng = np.random.Generator(np.random.PCG64(seed))
    xi = rng.uniform(-1.0, 1.0, size=rho0.shape)
    rho = rho0 * (1.0 + 0.01 * xi)
    p = BLOB_K * rho0 ** BLOB_GAMMA
    inside = r < BLOB_R
    Vx = np.where(inside, -BLOB_OMEGA * Y, 0.0)
    Vy = np.where(inside, BLOB_OMEGA * X, 0.0)
    # zero shift: Eulerian velocity v^i = V^i / alpha; W from gamma_ij = psi^4 delta_ij
    vx, vy = Vx / alp_c, Vy / alp_c
    W = 1.0 / np.sqrt(1.0 - psi4_c * (vx * vx + vy * vy))
    # poloidal field: A = f(r) (-y, x, 0), f = A_b q(r), q = max(p - 0.04 p_max, 0)
    pmax = BLOB_K * (BLOB_RHOC * (1.0 + BLOB_ATM)) ** BLOB_GAMMA
    q = np.maximum(p - 0.04 * pmax, 0.0)
    dpdr = BLOB_K * BLOB_GAMMA * rho0 ** (BLOB_GAMMA - 1.0) * BLOB_RHOC * (-2.0 * r / BLOB_R ** 2)
    dqdr = np.where((q > 0.0) & inside, dpdr, 0.0)
    with np.errstate(invalid="ignore", divide="ignore"):
        fr = np.where(r > 0, dqdr / r, 0.0)  # f'(r) / r
    curl_x = -X * Z * fr
    curl_y = -Y * Z * fr
    curl_z = 2.0 * q + (X * X + Y * Y) * fr
    # sqrt(gamma) Bn^i = curl A  ->  B^i = curl / (alpha sqrt(gamma)); sqrt(gamma) = psi^6
    sqrtgam = psi4_c ** 1.5
    Bx = curl_x / (alp_c * sqrtgam)
    By = curl_y / (alp_c * sqrtgam)
    Bz = curl_z / (alp_c * sqrtgam)
    # Eulerian field Bn = alpha B, |Bn|^2 = psi^4 |Bn|_flat^2 ; the field is poloidal and the
    # flow toroidal, so Bn.v = 0 and b^2 = Bn^2 / W^2.
    b2_unit = psi4_c * alp_c ** 2 * (Bx * Bx + By * By + Bz * Bz) / (W * W)
    Ab = math.sqrt(1e-3 * float(p.max()) / max(float((0.5 * b2_unit).max()), 1e-300))
    Bx, By, Bz = Ab * Bx, Ab * By, Ab * Bz
    if field == "toroidal":
        # Eulerian field alpha B^i = f e_phi^i with e_phi^i = (-y, x, 0) / (varpi psi^2), so that
        # gamma_ij (alpha B^i)(alpha B^j) = f^2
        B0 = math.e * TOROIDAL_B_GAUSS / GAUSS_PER_CODE_UNIT
        varpi = np.sqrt(X * X + Y * Y)
        with np.errstate(invalid="ignore", divide="ignore"):
            ex = np.where(varpi > 0, -Y / varpi, 0.0)
            ey = np.where(varpi > 0, X / varpi, 0.0)
        f = B0 * toroidal_profile(X, Y, Z)
        psi2 = np.sqrt(psi4_c)
        Bx = f * ex / (psi2 * alp_c)
        By = f * ey / (psi2 * alp_c)
        Bz = np.zeros_like(Bx)
    elif field != "poloidal":
        raise ValueError(f"unknown field {field!r}")
    prim = np.zeros((9,) + rho.shape)
    prim[0] = rho
    prim[1] = p
    prim[2] = W * vx
    prim[3] = W * vy
    prim[5] = Bx
    prim[6] = By
    prim[7] = Bz
    return Problem(name=f"blob3d_{n}" + ("" if field == "poloidal" else f"_{field}"), n=nn,
                   dx=(dx,) * 3, x0=x0, bc=(0, 0, 0),
                   gamma=BLOB_GAMMA, prim=np.ascontiguousarray(prim), metric=met,
                   t_end=0.0, cfl=0.5, cleaning=cleaning, ch=ch, kappa=kappa,
                   rho_floor=BLOB_ATM * BLOB_RHOC, rho_atm=10.0 * BLOB_ATM * BLOB_RHOC,
                   p_floor=1e-30, atm_K=BLOB_K, steps=steps)


# ------------------------------------------------------------------ ensemble of 1-D tubes
def ensemble(count: int = 512, seed: int = 1103, nmin: int = 200, nmax: int = 4000,
             t_end: float = 0.4) -> List[Problem]:
    """Independent magnetised tubes: N ~ U{200..4000}; rho, p log-uniform in [0.01, 10] with
    left/right ratios <= 1e3 (redrawn otherwise); v_x ~ U[-0.5, 0.5] per side; B_x ~ U[0, 1]
    shared; B_y, B_z ~ U[-2, 2] per side; Gamma uniform over {4/3, 5/3, 2}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gammas = (4.0 / 3.0, 5.0 / 3.0, 2.0)
    out = []
    for i in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        while True:
            rl, rr = 10 ** rng.uniform(-2, 1, size=2)
            pl, pr = 10 ** rng.uniform(-2, 1, size=2)
            if max(rl / rr, rr / rl) <= 1e3 and max(pl / pr, pr / pl) <= 1e3:
                break
        vxl, vxr = rng.uniform(-0.5, 0.5, size=2)
        bx = rng.uniform(0.0, 1.0)
        byl, byr, bzl, bzr = rng.uniform(-2.0, 2.0, size=4)
        gam = gammas[int(rng.integers(0, 3))]
        left = dict(rho=rl, p=pl, vx=vxl, Bx=bx, By=byl, Bz=bzl)
        right = dict(rho=rr, p=pr, vx=vxr, Bx=bx, By=byr, Bz=bzr)
        out.append(shock_tube(n, left, right, gam, t_end, name=f"tube{i}"))
    return out


# ------------------------------------------------------------------ pointwise random inputs
def random_metric_points(count: int, seed: int, strength: float = 0.3) -> np.ndarray:
    """(count, 10) metrics: alpha in [0.5, 1], |beta| <= 0.2, gamma_ij = a (I + s H) with H
    symmetric, entries in [-1, 1] scaled so that gamma stays positive definite."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.zeros((count, 10))
    out[:, 0] = rng.uniform(0.5, 1.0, count)
    out[:, 1:4] = rng.uniform(-0.2, 0.2, (count, 3)) / math.sqrt(3.0)
    for c in range(count):
        H = rng.uniform(-1.0, 1.0, (3, 3))
        H = 0.5 * (H + H.T)
        a = rng.uniform(1.0, 2.0)
        g = a * (np.eye(3) + strength * H / 3.0)
        out[c, 4:] = [g[0, 0], g[0, 1], g[0, 2], g[1, 1], g[1, 2], g[2, 2]]
    return out


def random_prim_points(count: int, seed: int, met: np.ndarray, wmax: float = 10.0,
                       sigma_max: float = 100.0, cleaning: bool = False) -> np.ndarray:
    """(count, 9) primitive states: rho in [1e-6, 10] (log), p/rho in [1e-4, 1e2] (log),
    Lorentz factor up to ``wmax``, magnetisation B_n^2 / rho up to ``sigma_max`` (log)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.zeros((count, 9))
    for c in range(count):
        rho = 10 ** rng.uniform(-6, 1)
        p = rho * 10 ** rng.uniform(-4, 2)
        g = np.array([[met[c, 4], met[c, 5], met[c, 6]],
                      [met[c, 5], met[c, 7], met[c, 8]],
                      [met[c, 6], met[c, 8], met[c, 9]]])
        dirn = rng.normal(size=3)
        dirn /= math.sqrt(float(dirn @ g @ dirn))       # unit length in gamma_ij
        W = 10 ** rng.uniform(0.0, math.log10(wmax))
        ut = math.sqrt(W * W - 1.0) * dirn              # gamma_ij u~^i u~^j = W^2 - 1
        bdir = rng.normal(size=3)
        bdir /= math.sqrt(float(bdir @ g @ bdir))
        sig = 10 ** rng.uniform(-4, math.log10(sigma_max))
        Bn = math.sqrt(sig * rho) * bdir                # Eulerian field alpha B^i
        B = Bn / met[c, 0]
        psi = rng.uniform(-0.1, 0.1) if cleaning else 0.0
        out[c] = [rho, p, ut[0], ut[1], ut[2], B[0], B[1], B[2], psi]
    return out


def smooth_periodic(n: Sequence[int], seed: int, amp: float = 0.1, magnetised: bool = True,
                    gamma: float = 5.0 / 3.0, L: float = 1.0) -> Problem:
    """Smooth random-phase periodic data on [0, L)^dims in Minkowski (conservation tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nn = tuple(int(k) for k in n)
    dx = tuple(L / k for k in nn)
    xs = centre_coords(nn, dx, (0.0, 0.0, 0.0), with_ghost=False)
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")

    def wave():
        k = [rng.integers(1, 3) if nn[d] > 1 else 0 for d in range(3)]
        ph = rng.uniform(0, 2 * math.pi)
        return np.sin(2 * math.pi * (k[0] * X + k[1] * Y + k[2] * Z) / L + ph)

    prim = np.zeros((9,) + X.shape)
    prim[0] = 1.0 + 0.5 * amp * wave()
    prim[1] = 1.0 + 0.5 * amp * wave()
    for f in (2, 3, 4):
        prim[f] = 0.3 + amp * wave()
    if magnetised:
        for f in (5, 6, 7):
            prim[f] = 0.5 + amp * wave()
    return Problem(name="smooth", n=nn, dx=dx, x0=(0.0, 0.0, 0.0), bc=(1, 1, 1), gamma=gamma,
                   prim=np.ascontiguousarray(prim), metric=minkowski_metric(nn))


def with_periodic_metric(prob: Problem, met_fn) -> Problem:
    """Replace the metric by ``met_fn(X, Y, Z) -> (10, ...)`` evaluated at centres with the
    ghost layer wrapped periodically (for periodic problems in a curved static metric)."""
    nn, dx = prob.n, prob.dx
    gx = metric_ghosts(nn)
    axes = []
    for d in range(3):
        idx = np.arange(-gx[d], nn[d] + gx[d]) % nn[d]
        axes.append(prob.x0[d] + (idx + 0.5) * dx[d])
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    prob.metric = np.ascontiguousarray(met_fn(X, Y, Z))
    return prob


# ------------------------------------------------------------------ gradient (adjoint) workloads
# The 1-D inverse problem: the initial state of the magnetised shock tube is described by ten
# left / right parameters and an additive density perturbation per cell; the loss is the L2
# misfit of the final density against a target profile.  B^x is not a parameter: a jump in it
# would violate the divergence constraint (§2.1).
#
# Base point.  On an exactly uniform state every limited slope sits on the kink of |x|, and in
# the tails of the waves neighbouring cells differ by a few ulps, so the frozen-branch
# derivative there depends on rounding: per-cell gradients of an untextured tube differ by
# percents between two correct implementations (FMA contraction alone does it).  The base
# point of the per-cell density parameters is therefore a seeded texture of relative size 1e-3,
# and a fixed seeded texture of the same size is added to p, u~^i, B^y and B^z; B^x stays
# uniform (its slopes are exactly zero and stay so).  Derivatives at this generic point agree
# between implementations to round-off.
TUBE_PARAM_NAMES = ("rho_L", "p_L", "vx_L", "By_L", "Bz_L", "rho_R", "p_R", "vx_R", "By_R", "Bz_R")
TUBE_PARAMS_DEFAULT = np.array([1.0, 1.0, 0.0, 1.0, 0.0, 0.125, 0.1, 0.0, -1.0, 0.0])
TUBE_BX = 0.5
TUBE_TEXTURE = 1e-3


def tube_texture(n: int, seed: int = 1104, amp: float = TUBE_TEXTURE) -> np.ndarray:
    """(9, n): row 0 is the base value of the per-cell density perturbation (relative to the
    side's density); rows 1-4, 6, 7 the fixed additive texture of p (relative to the side's
    pressure), u~^x, u~^y, u~^z, B^y, B^z; rows 5 (B^x) and 8 (psi) are zero."""
    rng = np.random.default_rng(seed)
    left = (np.arange(n) + 0.5) / n < 0.5
    t = np.zeros((9, n))
    if amp == 0.0:
        return t
    t[0] = amp * np.where(left, TUBE_PARAMS_DEFAULT[0], TUBE_PARAMS_DEFAULT[5]) * rng.standard_normal(n)
    t[1] = amp * np.where(left, TUBE_PARAMS_DEFAULT[1], TUBE_PARAMS_DEFAULT[6]) * rng.standard_normal(n)
    for f in (2, 3, 4, 6, 7):
        t[f] = amp * rng.standard_normal(n)
    return t


def tube_prim_from_params(theta, drho, n: int, xp=np, texture=None):
    """Primitives (9, 1, 1, n) of the tube on [-0.5, 0.5] from the ten parameters, the per-cell
    density perturbation drho (length n) and an optional fixed texture (rows 1-7 of
    tube_texture are added; row 0 is the base value of drho, not added here).  ``xp`` is numpy
    or torch (then the map is differentiable by autograd); u~^x = W v^x, W = 1/sqrt(1 - v^2)."""
    if xp is np:
        left = (np.arange(n) + 0.5) / n < 0.5
        sel = lambda a, b: np.where(left, a, b)
        zeros = np.zeros(n)
        stack = np.stack
        tex = texture
    else:
        left = (xp.arange(n, dtype=xp.float64, device=drho.device) + 0.5) / n < 0.5
        sel = lambda a, b: xp.where(left, a, b)
        zeros = xp.zeros(n, dtype=xp.float64, device=drho.device)
        stack = xp.stack
        tex = None if texture is None else xp.as_tensor(texture, dtype=xp.float64, device=drho.device)
    rho = sel(theta[0], theta[5]) + drho
    p = sel(theta[1], theta[6]) + zeros
    v = sel(theta[2], theta[7]) + zeros
    ut = v / xp.sqrt(1.0 - v * v)
    by = sel(theta[3], theta[8]) + zeros
    bz = sel(theta[4], theta[9]) + zeros
    bx = zeros + TUBE_BX
    uy, uz = zeros, zeros
    if tex is not None:
        p = p + tex[1]
        ut = ut + tex[2]
        uy = uy + tex[3]
        uz = uz + tex[4]
        by = by + tex[6]
        bz = bz + tex[7]
    prim = stack([rho, p, ut, uy, uz, bx, by, bz, zeros])
    return prim.reshape(9, 1, 1, n)


def adjoint_tube(n: int = 800, cfl: float = 0.4, steps: int = 1000, seed: int = 1104,
                 texture: float = TUBE_TEXTURE) -> Problem:
    """Gradient workload, 1-D: the tube of ``balsara1`` (Gamma = 2) at N cells at the textured
    base point above, ``steps`` fixed steps of size fixed_dt = cfl * dx (a light-speed bound,
    independent of the parameters)."""
    P = shock_tube(n, BALSARA1_LEFT, BALSARA1_RIGHT, 2.0, 0.0, name="adjoint_tube", cfl=cfl)
    tex = tube_texture(n, seed, texture)
    P.prim = np.ascontiguousarray(tube_prim_from_params(TUBE_PARAMS_DEFAULT, tex[0], n, texture=tex))
    P.steps = steps
    P.t_end = steps * cfl * P.dx[0]
    return P


def fixed_dt(P: Problem) -> float:
    """Fixed step of the gradient workloads: the light-speed bound of the unsplit update,
    dt = cfl / sum over active axes of 1/dx_d (the Courant numbers of the axes add up; with
    fast waves near c, dt = cfl * dx alone is linearly unstable in 2-D and the derivative of a
    long run grows without bound even though the state looks fine)."""
    return P.cfl / sum(1.0 / P.dx[d] for d in range(3) if P.n[d] > 1)


def blast2d(n: int = 256, half_width: float = 6.0, r_in: float = 0.8, rho_in: float = 0.01,
            p_in: float = 1.0, rho_out: float = 1e-4, p_out: float = 5e-4, bx: float = 0.1,
            gamma: float = 4.0 / 3.0, cfl: float = 0.4, steps: int = 200) -> Problem:
    """Gradient workload, 2-D: cylindrical magnetised blast wave on [-L, L]^2 (n^2 cells,
    Minkowski, outflow): rho_in, p_in inside r < r_in, ambient rho_out, p_out outside, uniform
    B^x, at rest; ``steps`` fixed steps of size fixed_dt (cfl * dx / 2)."""
    dx = 2.0 * half_width / n
    c = -half_width + (np.arange(n) + 0.5) * dx
    y, x = np.meshgrid(c, c, indexing="ij")
    inner = np.sqrt(x * x + y * y) < r_in
    prim = np.zeros((9, 1, n, n))
    prim[0, 0] = np.where(inner, rho_in, rho_out)
    prim[1, 0] = np.where(inner, p_in, p_out)
    prim[5, 0] = bx
    nn = (n, n, 1)
    return Problem(name="blast2d", n=nn, dx=(dx, dx, 1.0), x0=(-half_width, -half_width, 0.0),
                   bc=(0, 0, 0), gamma=gamma, prim=prim, metric=minkowski_metric(nn),
                   t_end=steps * 0.5 * cfl * dx, cfl=cfl, steps=steps)


def blast2d_inner_mask(P: Problem, r_in: float = 0.8) -> np.ndarray:
    """Cells of the blast wave's inner region (where the inner pressure parameter acts)."""
    n = P.n[0]
    c = P.x0[0] + (np.arange(n) + 0.5) * P.dx[0]
    y, x = np.meshgrid(c, c, indexing="ij")
    return (np.sqrt(x * x + y * y) < r_in)[None, :, :]


def tube_param_directions(theta, n: int):
    """d prim(0) / d theta_q for the ten tube parameters (analytic; du~/dv = W^3)."""
    left = (np.arange(n) + 0.5) / n < 0.5
    out = []
    for q in range(10):
        side = left if q < 5 else ~left
        k = q % 5
        d = np.zeros((9, 1, 1, n))
        field = (0, 1, 2, 6, 7)[k]
        val = 1.0
        if k == 2:
            v = theta[q]
            val = (1.0 - v * v) ** -1.5
        d[field, 0, 0, side] = val
        out.append(d)
    return out
