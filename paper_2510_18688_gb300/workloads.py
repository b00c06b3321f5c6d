"""Seeded synthetic inputs shaped like the paper's benchmarks (arXiv 2510.18688, Sec. 4).

This module only generates inputs: a parameter dictionary (physical and
lattice-unit parameters, the same keys for the CUDA library and for the test
oracle) and the initial arrays ``phi0`` (pre-existing solid), ``phi`` (order
parameter), ``T`` (temperature), ``fl`` (liquid fraction) and an optional
cold ``mask``.  It holds none of the method's arithmetic: the geometry is
built from the initial profiles the paper prints (Eqs. (34) and (38)) and
random numbers from ``numpy.random.Generator(PCG64(seed))``.

Arrays are ``[ny, nx]`` float64, x fastest.  Node ``(i, j)`` sits at the
physical position ``(i + 1/2, j + 1/2)`` measured from the lower-left walls,
which sit half-way between the first node and its ghost.

Parameter conventions (lattice units, dx = dt = 1, T_m = 0):

* ``lattices``: bit 0 flow, bit 1 phase field, bit 2 enthalpy.
* ``bc``: ``(x_lo, x_hi, y_lo, y_hi)``, each ``"periodic"``, ``"dirichlet"``
  (no-slip, no-flux, fixed temperature ``T_wall[k]``) or ``"adiabatic"``.
* ``latent`` is L; it follows from the Stefan number of Eq. (29),
  Ste = Cp_l (T_m - T_w) / L.
* Gas properties follow the reading R-GAS: equal kinematic viscosity, equal
  conductivity and equal volumetric heat capacity as the liquid (the last is
  what keeps the rest population of the enthalpy lattice positive).
* The gas/liquid density ratio defaults to 0.1: at 0.001 a gas-liquid
  interface that moves normal to itself is unstable in this method as read
  (a translating flat interface in a periodic box diverges within a few
  thousand steps even at u = 1e-5), so every moving-interface workload uses
  0.1 unless a caller overrides ``rho_g``.
"""
from __future__ import annotations

import math

import numpy as np

FLOW, PHASE, HEAT = 1, 2, 4
ALL = FLOW | PHASE | HEAT


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def latent_from_stefan(ste: float, cp_l: float = 1.0, T_w: float = -1.0) -> float:
    """L from Ste = Cp_l (T_m - T_w) / L with T_m = 0 (Eq. (29))."""
    return cp_l * (0.0 - T_w) / ste


def base_params(nx: int, ny: int, **kw) -> dict:
    """Default parameter set; every key may be overridden."""
    rho_l = kw.pop("rho_l", 1.0)
    rho_s = kw.pop("rho_s", 0.9)
    rho_g = kw.pop("rho_g", 0.1)
    nu = kw.pop("nu", 0.1)
    cp_l = kw.pop("cp_l", 1.0)
    cp_s = kw.pop("cp_s", 1.0)
    lam_l = kw.pop("lambda_l", 0.1)
    p = dict(
        nx=int(nx), ny=int(ny), lattices=ALL,
        bc=("periodic", "periodic", "periodic", "periodic"),
        T_wall=(0.0, 0.0, 0.0, 0.0),
        rho_l=rho_l, rho_s=rho_s, rho_g=rho_g,
        mu_l=rho_l * nu, mu_s=rho_l * nu, mu_g=rho_g * nu,
        lambda_l=lam_l, lambda_s=lam_l, lambda_g=lam_l,
        cp_l=cp_l, cp_s=cp_s, cp_g=cp_l * rho_l / rho_g,
        rho_ref=rho_l, latent=latent_from_stefan(0.1, cp_l),
        sigma=0.001, eps=4.0, mobility=0.1, eta=1.0,
        theta_deg=90.0, psi_deg=90.0,
        gx=0.0, gy=0.0, T_cold=-1.0, readings=0,
    )
    p.update(kw)
    return p


def _grid(nx: int, ny: int):
    x = np.arange(nx, dtype=np.float64) + 0.5
    y = np.arange(ny, dtype=np.float64) + 0.5
    return np.meshgrid(x, y)  # each [ny, nx]


def _arrays(phi0, phi, T, fl, mask=None) -> dict:
    a = dict(phi0=np.ascontiguousarray(phi0, dtype=np.float64),
             phi=np.ascontiguousarray(phi, dtype=np.float64),
             T=np.ascontiguousarray(T, dtype=np.float64),
             fl=np.ascontiguousarray(fl, dtype=np.float64))
    if mask is not None:
        a["mask"] = np.ascontiguousarray(mask, dtype=np.uint8)
    return a


# ---------------------------------------------------------------------------
# Sec. 4.1: conduction-induced freezing in a semi-infinite space
# ---------------------------------------------------------------------------

def neumann(nx=400, ny=4, T0=0.1, T_b=-1.0, ste=0.1, alpha=0.2, lambda_ratio=1.0,
            rho_ratio=1.0, nu=0.1):
    """Liquid at T0 >= T_m, cold Dirichlet wall T_b at x = 0, far wall at T0,
    periodic in y; flow and enthalpy lattices, phase field off (phi = 1)."""
    L = latent_from_stefan(ste, 1.0, T_b)
    p = base_params(nx, ny, rho_s=rho_ratio, nu=nu, lambda_l=alpha,
                    lattices=FLOW | HEAT, latent=L,
                    bc=("dirichlet", "dirichlet", "periodic", "periodic"),
                    T_wall=(T_b, T0, 0.0, 0.0))
    p["lambda_s"] = alpha * lambda_ratio
    z = np.zeros((ny, nx))
    return p, _arrays(z, z + 1.0, z + T0, z + 1.0)


# ---------------------------------------------------------------------------
# Sec. 4.2: three-phase Stefan problem with volume change (Eq. (34))
# ---------------------------------------------------------------------------

def stefan(nx=512, ny=8, hs=16.0, h0=80.0, rho_ratio=0.9, ste=0.1, alpha=0.5,
           T0=1.0, T_b=-1.0, eps=4.0):
    """Solid layer (phi0) below x = hs, liquid up to x = h0, gas above;
    walls in x (cold T_b at x = 0, T0 at the far end), periodic in y."""
    p = base_params(nx, ny, rho_s=rho_ratio, lambda_l=alpha, eps=eps, sigma=0.001,
                    mobility=0.1, nu=0.1, latent=latent_from_stefan(ste, 1.0, T_b),
                    bc=("dirichlet", "dirichlet", "periodic", "periodic"),
                    T_wall=(T_b, T0, 0.0, 0.0))
    X, _ = _grid(nx, ny)
    phi0 = 0.5 + 0.5 * np.tanh(2.0 * (hs - X) / eps)
    phi = (1.0 - phi0) * np.tanh(2.0 * (h0 - X) / eps)
    z = np.zeros((ny, nx))
    return p, _arrays(phi0, phi, z + T0, z + 1.0)


# ---------------------------------------------------------------------------
# Sec. 4.3: sessile droplet on a flat cold substrate
# ---------------------------------------------------------------------------

def sessile_droplet(n=512, seed=0, radius=100.0, hs=12.0, T0=0.1, T_w=-1.0,
                    theta_deg=None, ste=None, rho_ratio=0.9, eps=4.0, ny=None):
    """Circular cap of radius R at contact angle theta on a solid layer of
    height hs (cold mask at T_w); periodic in x, walls in y.  theta and Ste
    are drawn from U[60, 120] degrees and U[0.1, 0.5] unless given."""
    r = rng(seed)
    th = float(r.uniform(60.0, 120.0)) if theta_deg is None else float(theta_deg)
    st = float(r.uniform(0.1, 0.5)) if ste is None else float(ste)
    nx = n
    ny = n if ny is None else ny
    p = base_params(nx, ny, rho_s=rho_ratio, cp_s=0.5, lambda_l=0.1, eps=eps,
                    latent=latent_from_stefan(st, 1.0, T_w), theta_deg=th, T_cold=T_w,
                    bc=("periodic", "periodic", "dirichlet", "adiabatic"),
                    T_wall=(0.0, 0.0, T_w, 0.0))
    p["lambda_s"] = 0.37
    X, Y = _grid(nx, ny)
    phi0 = 0.5 + 0.5 * np.tanh(2.0 * (hs - Y) / eps)
    yc = hs - radius * math.cos(math.radians(th))
    d = np.hypot(X - nx / 2.0, Y - yc)
    phi = (1.0 - phi0) * np.tanh(2.0 * (radius - d) / eps)
    mask = phi0 >= 0.5
    T = np.where(mask, T_w, T0)
    fl = np.where(T < 0.0, 0.0, 1.0)
    return p, _arrays(phi0, phi, T, fl, mask)


# ---------------------------------------------------------------------------
# Sec. 4.4: droplet on a cold cylinder (Eq. (38))
# ---------------------------------------------------------------------------

def cylinder_droplet(side=256, seed=0, T0=0.1, T_w=-1.0, eps=4.0):
    """Cylinder of radius Rs = U[0.2, 0.4] side at (L/2, L/4) as cold solid
    mask, droplet R0 = Rs/2 on top, theta ~ U[30, 150], Ste ~ U[0.05, 0.5]."""
    r = rng(seed)
    rs = float(r.uniform(0.2, 0.4)) * side
    th = float(r.uniform(30.0, 150.0))
    st = float(r.uniform(0.05, 0.5))
    r0 = 0.5 * rs
    p = base_params(side, side, cp_s=0.5, lambda_l=0.1, eps=eps,
                    latent=latent_from_stefan(st, 1.0, T_w), theta_deg=th, T_cold=T_w,
                    bc=("periodic", "periodic", "adiabatic", "adiabatic"))
    p["lambda_s"] = 0.37
    X, Y = _grid(side, side)
    dc = np.hypot(X - side / 2.0, Y - side / 4.0)
    phi0 = 0.5 + 0.5 * np.tanh((rs - dc) / (eps / 2.0))
    dd = np.hypot(X - side / 2.0, Y - side / 4.0 - rs)
    phi = (1.0 - phi0) * np.tanh((r0 - dd) / (eps / 2.0))
    mask = phi0 >= 0.5
    T = np.where(mask, T_w, T0)
    fl = np.where(T < 0.0, 0.0, 1.0)
    return p, _arrays(phi0, phi, T, fl, mask)


# ---------------------------------------------------------------------------
# Sec. 4.6: unsaturated porous medium (synthetic stand-in for the sandpack)
# ---------------------------------------------------------------------------

def _disks(r, nx, ny, target_cover, rmin, rmax, gap, max_tries=200000):
    """Random sequential addition of non-overlapping disks (centres, radii)."""
    cs, rs = [], []
    area = 0.0
    tries = 0
    while area < target_cover * nx * ny and tries < max_tries:
        tries += 1
        rad = r.uniform(rmin, rmax)
        cx, cy = r.uniform(0, nx), r.uniform(0, ny)
        if cs:
            c = np.asarray(cs)
            dx = np.abs(c[:, 0] - cx)
            dx = np.minimum(dx, nx - dx)  # periodic distance in x only for spacing
            dy = c[:, 1] - cy
            if np.any(np.hypot(dx, dy) < np.asarray(rs) + rad + gap):
                continue
        cs.append((cx, cy))
        rs.append(rad)
        area += math.pi * rad * rad
    return np.asarray(cs), np.asarray(rs)


def _signed_distance_to_disks(X, Y, centres, radii, chunk=64):
    """max over disks of (radius - distance): > 0 inside a disk."""
    best = np.full(X.shape, -1e30)
    for k in range(0, len(radii), chunk):
        c = centres[k:k + chunk]
        rr = radii[k:k + chunk]
        for (cx, cy), rad in zip(c, rr):
            best = np.maximum(best, rad - np.hypot(X - cx, Y - cy))
    return best


def porous(nx=2048, ny=1024, seed=0, porosity=0.6, saturation=0.5, eps=4.0,
           theta_deg=60.0, T_b=-1.0, T_w=0.1, ste=0.1):
    """Random non-overlapping circular grains (r ~ U[10, 30], gap 2 eps) to the
    given porosity; liquid blobs in the pore space to the given saturation;
    cold wall at x = 0, warm wall at x = nx, adiabatic walls in y."""
    r = rng(seed)
    X, Y = _grid(nx, ny)
    gc, gr = _disks(r, nx, ny, 1.0 - porosity, 10.0, 30.0, 2.0 * eps)
    dg = _signed_distance_to_disks(X, Y, gc, gr)
    phi0 = 0.5 + 0.5 * np.tanh(2.0 * dg / eps)
    pore = phi0 < 0.5
    pore_area = float(pore.sum())
    # liquid blobs: random disks in the pore space until the saturation is met
    lc, lr = [], []
    liquid = np.zeros_like(pore)
    tries = 0
    while liquid.sum() < saturation * pore_area and tries < 100000:
        tries += 1
        rad = r.uniform(8.0, 40.0)
        cx, cy = r.uniform(0, nx), r.uniform(0, ny)
        lc.append((cx, cy))
        lr.append(rad)
        liquid |= (np.hypot(X - cx, Y - cy) < rad) & pore
    dl = _signed_distance_to_disks(X, Y, np.asarray(lc), np.asarray(lr))
    phi = (1.0 - phi0) * np.tanh(2.0 * dl / eps)
    p = base_params(nx, ny, cp_s=1.0, lambda_l=0.1, eps=eps, theta_deg=theta_deg,
                    latent=latent_from_stefan(ste, 1.0, T_b),
                    bc=("dirichlet", "dirichlet", "adiabatic", "adiabatic"),
                    T_wall=(T_b, T_w, 0.0, 0.0))
    p["lambda_s"] = 0.37
    T = np.full((ny, nx), T_w)
    fl = np.ones((ny, nx))
    return p, _arrays(phi0, phi, T, fl)


# ---------------------------------------------------------------------------
# generic seeded states for parity tests
# ---------------------------------------------------------------------------

def random_state(nx, ny, seed=0, lattices=ALL, bc=None, n_blobs=3, mushy=True):
    """Small seeded three-phase state that exercises every branch: solid
    blobs (phi0), liquid drops and gas, temperatures on both sides of T_m
    (with mushy nodes), random contact angle, gravity and cold mask."""
    r = rng(seed)
    if bc is None:
        bc = [("periodic", "periodic", "dirichlet", "adiabatic"),
              ("dirichlet", "adiabatic", "periodic", "periodic"),
              ("periodic", "periodic", "periodic", "periodic"),
              ("dirichlet", "dirichlet", "adiabatic", "dirichlet")][seed % 4]
    X, Y = _grid(nx, ny)
    eps = 4.0
    per_x, per_y = bc[0] == "periodic", bc[2] == "periodic"

    def dist(cx, cy):
        # minimum-image distance on periodic axes keeps the fields smooth
        dx, dy = np.abs(X - cx), np.abs(Y - cy)
        if per_x:
            dx = np.minimum(dx, nx - dx)
        if per_y:
            dy = np.minimum(dy, ny - dy)
        return np.hypot(dx, dy)

    phi0 = np.zeros((ny, nx))
    dl = np.full((ny, nx), -1e30)
    for _ in range(n_blobs):
        cx, cy = r.uniform(0, nx), r.uniform(0, ny)
        rad = r.uniform(2.0, max(3.0, min(nx, ny) / 4.0))
        phi0 = np.maximum(phi0, 0.5 + 0.5 * np.tanh(2.0 * (rad - dist(cx, cy)) / eps))
        cx, cy = r.uniform(0, nx), r.uniform(0, ny)
        rad = r.uniform(3.0, max(4.0, min(nx, ny) / 3.0))
        dl = np.maximum(dl, rad - dist(cx, cy))
    phi = (1.0 - phi0) * np.tanh(2.0 * dl / eps)
    T = 0.3 * np.sin(2 * np.pi * X / nx * r.integers(1, 3)) + 0.2 * r.standard_normal() \
        + 0.05 * np.cos(2 * np.pi * Y / ny)  # periodic in both axes
    # pre-existing ice only well inside the liquid: frozen material next to
    # gas at t = 0 is far from the phase-field equilibrium of Eq. (4)
    T = np.where(phi < 0.9, np.maximum(T, 0.1), T)
    fl = np.where(T < 0.0, 0.0, 1.0)
    if mushy:
        # a smooth mushy band: T = T_m and fl rising from 0 to 1 across it
        band = np.abs(T) < 0.05
        fl = np.where(band, 0.5 + T / 0.1, fl)
        T = np.where(band, 0.0, T)
    mask = (phi0 > 0.7) & (r.uniform(size=phi0.shape) < 0.5)
    p = base_params(nx, ny, rho_s=float(r.uniform(0.85, 1.1)), cp_s=0.8, lambda_l=0.12,
                    latent=latent_from_stefan(float(r.uniform(0.1, 0.5))),
                    theta_deg=float(r.uniform(40.0, 140.0)),
                    psi_deg=float(r.uniform(70.0, 110.0)),
                    gx=float(r.uniform(-1e-6, 1e-6)), gy=float(r.uniform(-1e-6, 1e-6)),
                    bc=bc, T_wall=tuple(float(v) for v in r.uniform(-1.0, 0.5, size=4)),
                    T_cold=-0.8, lattices=lattices)
    p["lambda_s"] = 0.3
    return p, _arrays(phi0, phi, T, fl, mask)


# ---------------------------------------------------------------------------
# three-dimensional (D3Q19) inputs: arrays are [nz, ny, nx], x fastest; the
# parameter dictionary adds nz, gz, and six boundary types and wall
# temperatures (x_lo, x_hi, y_lo, y_hi, z_lo, z_hi)
# ---------------------------------------------------------------------------

def extrude_z(wl, nz: int):
    """A two-dimensional workload repeated along a periodic z axis."""
    cfg, arr = wl
    p = dict(cfg, nz=int(nz), gz=0.0, bc=tuple(cfg["bc"]) + ("periodic", "periodic"),
             T_wall=tuple(cfg["T_wall"]) + (0.0, 0.0))
    out = {k: np.ascontiguousarray(np.broadcast_to(v, (nz,) + v.shape)) for k, v in arr.items()}
    return p, out


def _grid3(nx: int, ny: int, nz: int):
    x = np.arange(nx, dtype=np.float64) + 0.5
    y = np.arange(ny, dtype=np.float64) + 0.5
    z = np.arange(nz, dtype=np.float64) + 0.5
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")  # each [nz, ny, nx]
    return X, Y, Z


def random_state3(nx, ny, nz, seed=0, lattices=ALL, bc=None, n_blobs=3, mushy=True):
    """Small seeded three-phase state in 3-D that exercises every branch, as
    random_state does in 2-D: solid blobs, liquid drops and gas, temperatures
    on both sides of T_m with mushy nodes, random contact angle, gravity in
    all three axes and a cold mask."""
    r = rng(seed)
    if bc is None:
        bc = [("periodic", "periodic", "periodic", "periodic", "dirichlet", "adiabatic"),
              ("dirichlet", "adiabatic", "periodic", "periodic", "periodic", "periodic"),
              ("periodic", "periodic", "periodic", "periodic", "periodic", "periodic"),
              ("dirichlet", "dirichlet", "adiabatic", "dirichlet", "adiabatic", "adiabatic")][seed % 4]
    X, Y, Z = _grid3(nx, ny, nz)
    eps = 4.0
    per = (bc[0] == "periodic", bc[2] == "periodic", bc[4] == "periodic")

    def dist(cx, cy, cz):
        d = []
        for V, c, n, pr in ((X, cx, nx, per[0]), (Y, cy, ny, per[1]), (Z, cz, nz, per[2])):
            a = np.abs(V - c)
            d.append(np.minimum(a, n - a) if pr else a)
        return np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)

    shape = (nz, ny, nx)
    m = min(nx, ny, nz)
    # draw until the state has every branch (solid, liquid and gas; liquid
    # below and above T_m; a mushy band when asked for; masked nodes), at
    # most 64 times (the smallest grids cannot hold them all)
    for _attempt in range(64):
        phi0 = np.zeros(shape)
        dl = np.full(shape, -1e30)
        for _ in range(n_blobs):
            c = (r.uniform(0, nx), r.uniform(0, ny), r.uniform(0, nz))
            rad = r.uniform(2.0, max(3.0, m / 3.0))
            phi0 = np.maximum(phi0, 0.5 + 0.5 * np.tanh(2.0 * (rad - dist(*c)) / eps))
            c = (r.uniform(0, nx), r.uniform(0, ny), r.uniform(0, nz))
            rad = r.uniform(3.0, max(4.0, m / 2.0))
            dl = np.maximum(dl, rad - dist(*c))
        phi = (1.0 - phi0) * np.tanh(2.0 * dl / eps)
        T = (0.3 * np.sin(2 * np.pi * X / nx * r.integers(1, 3)) + 0.2 * r.standard_normal()
             + 0.05 * np.cos(2 * np.pi * Y / ny) + 0.05 * np.sin(2 * np.pi * Z / nz))
        T = np.where(phi < 0.9, np.maximum(T, 0.1), T)
        fl = np.where(T < 0.0, 0.0, 1.0)
        band = np.abs(T) < 0.05
        if mushy:
            fl = np.where(band, 0.5 + T / 0.1, fl)
            T = np.where(band, 0.0, T)
        mask = (phi0 > 0.7) & (r.uniform(size=shape) < 0.5)
        complete = ((phi0 > 0.5).any() and (phi > 0.5).any() and (phi < -0.5).any()
                    and (T < 0.0).any() and (T > 0.0).any() and mask.any()
                    and (band.any() or not mushy))
        if complete:
            break
    p = base_params(nx, ny, rho_s=float(r.uniform(0.85, 1.1)), cp_s=0.8, lambda_l=0.12,
                    latent=latent_from_stefan(float(r.uniform(0.1, 0.5))),
                    theta_deg=float(r.uniform(40.0, 140.0)),
                    psi_deg=float(r.uniform(70.0, 110.0)),
                    gx=float(r.uniform(-1e-6, 1e-6)), gy=float(r.uniform(-1e-6, 1e-6)),
                    bc=bc, T_wall=tuple(float(v) for v in r.uniform(-1.0, 0.5, size=6)),
                    T_cold=-0.8, lattices=lattices)
    p["nz"] = int(nz)
    p["gz"] = float(r.uniform(-1e-6, 1e-6))
    p["lambda_s"] = 0.3
    return p, _arrays(phi0, phi, T, fl, mask)


def _self_affine_pair(r, n: int, std: float, hurst: float, mismatch: float):
    """Two periodic n x n rough surfaces with standard deviation std whose
    Fourier modes share phases at wavelengths longer than `mismatch` and are
    independent below it (spectral synthesis of a self-affine surface with
    Hurst exponent H: amplitude ~ k^-(1+H))."""
    k = np.fft.fftfreq(n) * n
    KX, KY = np.meshgrid(k, k)
    kk = np.hypot(KX, KY)
    amp = np.where(kk > 0, np.maximum(kk, 1e-12) ** (-(1.0 + hurst)), 0.0)
    ph_shared = r.uniform(0, 2 * np.pi, size=(n, n))
    ph_own = r.uniform(0, 2 * np.pi, size=(2, n, n))
    long_wave = kk < n / mismatch
    out = []
    for s in range(2):
        ph = np.where(long_wave, ph_shared, ph_own[s])
        h = np.real(np.fft.ifft2(amp * np.exp(1j * ph)))
        out.append(h / h.std() * std)
    return out


def rough_fracture(nx=256, ny=128, nz=30, seed=0, fd=2.25, std=2.5, mismatch=30.0,
                   aperture=12.0, theta_deg=60.0, T0=0.1, T_w=-1.0, ste=0.1, eps=4.0):
    """Freezing in a rough fracture (Sec. 4.5 shape): a 128-wide self-affine
    fracture of fractal dimension fd (Hurst exponent 3 - fd), standard
    deviation std and mismatch length `mismatch`, repeated once along x; the
    solid (phi0) lies outside the aperture along z.  A liquid column fills
    x < 0.75 Lx with three gas bubbles of radii 0.075, 0.05 and 0.01 Lx at
    (0.25, 0.25, 0.5), (0.5, 0.5, 0.5) and (0.25, 0.75, 0.5) (Lx, Ly, Lz);
    T = T0 everywhere, the wall at x = 0 at T_w (the far wall adiabatic),
    periodic in y and z.  The fracture surfaces are synthetic stand-ins for
    the paper's generated fractures, from numpy's seeded generator."""
    r = rng(seed)
    tile = ny
    lo, hi = _self_affine_pair(r, tile, std, 3.0 - fd, mismatch)
    reps = -(-nx // tile)
    lo = np.tile(lo, (1, reps))[:, :nx]   # [ny, nx]
    hi = np.tile(hi, (1, reps))[:, :nx]
    zc = nz / 2.0
    z_lo = zc - aperture / 2.0 + lo
    z_hi = np.maximum(zc + aperture / 2.0 + hi, z_lo + 2.0)
    X, Y, Z = _grid3(nx, ny, nz)
    d_solid = np.maximum(z_lo[None] - Z, Z - z_hi[None])  # > 0 inside the rock
    phi0 = 0.5 + 0.5 * np.tanh(2.0 * d_solid / eps)
    Lx, Ly, Lz = float(nx), float(ny), float(nz)
    dl = 0.75 * Lx - X
    for (cx, cy, cz), rad in (((0.25, 0.25, 0.5), 0.075), ((0.5, 0.5, 0.5), 0.05),
                              ((0.25, 0.75, 0.5), 0.01)):
        d = np.sqrt((X - cx * Lx) ** 2 + (Y - cy * Ly) ** 2 + (Z - cz * Lz) ** 2)
        dl = np.minimum(dl, d - rad * Lx)
    phi = (1.0 - phi0) * np.tanh(2.0 * dl / eps)
    p = base_params(nx, ny, rho_s=0.9, cp_s=0.5, lambda_l=0.1, eps=eps, theta_deg=theta_deg,
                    latent=latent_from_stefan(ste, 1.0, T_w), T_cold=T_w,
                    bc=("dirichlet", "adiabatic", "periodic", "periodic", "periodic", "periodic"),
                    T_wall=(T_w, 0.0, 0.0, 0.0, 0.0, 0.0))
    p["lambda_s"] = 0.37
    p["nz"] = int(nz)
    p["gz"] = 0.0
    shape = (nz, ny, nx)
    return p, _arrays(phi0, phi, np.full(shape, T0), np.ones(shape))
