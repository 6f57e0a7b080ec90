"""Seeded synthetic inputs for the MPDATA step.

This module is shared by the CPU oracle tests and the CUDA path; it holds none
of the advection scheme's arithmetic (no fluxes, ratios or limiter), only the
construction of the fields the scheme is applied to:

* tracer fields psi (cell centres),
* G-weighted Courant numbers U, V, W on the staggered faces i+1/2, j+1/2,
  k+1/2 (the C-grid convention of Sec. 3.1.4.1: u(i) sits half a cell to the
  right of q(i)),
* the metric/density field G (cell centres).

Every array is returned as an *interior* float64 array of shape (nz, ny, nx),
i fastest.  ``pad`` embeds an interior array in the halo-padded storage
[nz+2h][ny+2h][nx+2h] that the library and the oracle both use; the halo is
left at ``fill`` (it is never trusted as input by either side).

Horizontal flows are built from a stream function sampled at cell corners, so
that the discrete G-weighted divergence of (U, V) is exactly zero up to
rounding; vertical motion, where present, is either a prescribed weak
sinusoid (divergent) or comes from an x-z stream function (non-divergent).
The top face (k = nz-1/2) of W is always zero: the vertical boundaries carry
no flux.

Random numbers come from numpy's PCG64 (``numpy.random.default_rng(seed)``);
the default seed is 1234.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

DEFAULT_SEED = 1234


@dataclasses.dataclass
class Case:
    """One MPDATA problem: fields plus the scheme options it is run with."""
    name: str
    nx: int
    ny: int
    nz: int
    psi: np.ndarray          # (nz, ny, nx) or (ntracers, nz, ny, nx)
    u: np.ndarray            # (nz, ny, nx): face i+1/2
    v: np.ndarray            # (nz, ny, nx): face j+1/2
    w: np.ndarray            # (nz, ny, nx): face k+1/2 (top row is zero)
    g: np.ndarray            # (nz, ny, nx): cell centres, > 0
    iord: int = 2
    nonosc: int = 1
    steps: int = 1
    halo: int = 2
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def npoints(self) -> int:
        return self.nx * self.ny * self.nz


def pad(a: np.ndarray, h: int, fill: float = 0.0, dtype=np.float64) -> np.ndarray:
    """Embed an interior array (..., nz, ny, nx) into halo-padded storage."""
    a = np.asarray(a)
    shape = a.shape[:-3] + tuple(s + 2 * h for s in a.shape[-3:])
    out = np.full(shape, fill, dtype=dtype)
    out[..., h:h + a.shape[-3], h:h + a.shape[-2], h:h + a.shape[-1]] = a
    return np.ascontiguousarray(out)


def interior(a: np.ndarray, h: int) -> np.ndarray:
    """Inverse of ``pad``: the interior view of a padded array."""
    return a[..., h:a.shape[-3] - h, h:a.shape[-2] - h, h:a.shape[-1] - h]


# --------------------------------------------------------------------------
# flows from corner stream functions
# --------------------------------------------------------------------------

def _uv_from_corner_streamfunction(psi_c: np.ndarray):
    """(U, V) on faces from a stream function at corners (i+1/2, j+1/2).

    psi_c[k, j, i] is the value at the corner (i+1/2, j+1/2) of level k.
    U(i+1/2, j) = -(psi_c(i+1/2, j+1/2) - psi_c(i+1/2, j-1/2)),
    V(i, j+1/2) =   psi_c(i+1/2, j+1/2) - psi_c(i-1/2, j+1/2),
    periodic in i and j, so each cell's net outflow cancels exactly.
    """
    u = -(psi_c - np.roll(psi_c, 1, axis=-2))
    v = psi_c - np.roll(psi_c, 1, axis=-1)
    return u, v


def outflow_courant_max(u, v, w, g, kbc: int = 0) -> float:
    """Largest per-cell outflow Courant sum (a validity bound on the inputs).

    For cell c it is the sum over the three directions of the outward-pointing
    face values, divided by G_c; the donor-cell pass keeps psi >= 0 when it is
    at most 1.  W's bottom face (k-1/2 at k=0) is the zero boundary, or with
    kbc = 1 (periodic k) the top face.
    """
    u_m = np.roll(u, 1, axis=-1)
    v_m = np.roll(v, 1, axis=-2)
    if kbc == 1:
        w_m = np.roll(w, 1, axis=-3)
    else:
        w_m = np.concatenate([np.zeros_like(w[..., :1, :, :]), w[..., :-1, :, :]], axis=-3)
    out = (np.maximum(u, 0) - np.minimum(u_m, 0) + np.maximum(v, 0) - np.minimum(v_m, 0)
           + np.maximum(w, 0) - np.minimum(w_m, 0))
    return float(np.max(out / g))


# --------------------------------------------------------------------------
# configuration generators
# --------------------------------------------------------------------------

def rotation_2d(n: int = 64, seed: int = DEFAULT_SEED, steps: int = 100,
                courant: float = 0.5, radius_frac: float = 30.0 / 64.0,
                cone_height: float = 4.0, cone_radius: float = 8.0,
                cone_offset: float = 16.0, background: float = 1.0) -> Case:
    """2D solid-body rotation of a cone (Smolarkiewicz-style test), nz = 1.

    Rotation about the domain centre with the corner stream function
    Psi = 0.5 * omega * min(r, R)^2, R = radius_frac * n (30 cells at n = 64),
    omega = courant / R so the largest Courant number is about ``courant``;
    the flow vanishes outside R, so Psi is periodic and (U, V) is exactly
    non-divergent.  G = 1.  The cone (height 4, radius 8 cells) sits on a
    background of 1, its centre ``cone_offset`` cells from the rotation
    centre at an angle drawn from the seed.
    """
    rng = np.random.default_rng(seed)
    R = radius_frac * n
    omega = courant / R
    xc = yc = n / 2.0
    # corners at (i+1, j+1) in cell units (cell i spans [i, i+1])
    xi = np.arange(n) + 1.0
    X, Y = np.meshgrid(xi, xi, indexing="xy")   # Y[j, i], X[j, i]
    r2 = np.minimum((X - xc) ** 2 + (Y - yc) ** 2, R * R)
    psi_c = 0.5 * omega * r2
    u, v = _uv_from_corner_streamfunction(psi_c[None])
    w = np.zeros_like(u)
    g = np.ones_like(u)
    ang = rng.uniform(0.0, 2.0 * math.pi)
    cx = xc + cone_offset * math.cos(ang)
    cy = yc + cone_offset * math.sin(ang)
    xcell = np.arange(n) + 0.5
    Xc, Yc = np.meshgrid(xcell, xcell, indexing="xy")
    d = np.sqrt((Xc - cx) ** 2 + (Yc - cy) ** 2)
    psi = background + cone_height * np.maximum(0.0, 1.0 - d / cone_radius)
    return Case("rotation_2d", n, n, 1, psi[None].copy(), u, v, w, g,
                iord=2, nonosc=1, steps=steps, halo=2,
                meta=dict(omega=omega, R=R, cone_centre=(cx, cy), seed=seed))


def latlon_geometry(nx: int, ny: int, nz: int):
    """Cell-centre longitude/latitude of the lat-lon mapping and G = cos(lat).

    lambda_i = 2 pi (i+1/2)/nx, phi_j = -pi/3 + (2 pi/3)(j+1/2)/ny, so G lies
    in [0.5, 1] and 1/G stays bounded.
    """
    lam = 2.0 * math.pi * (np.arange(nx) + 0.5) / nx
    phi = -math.pi / 3.0 + (2.0 * math.pi / 3.0) * (np.arange(ny) + 0.5) / ny
    g = np.broadcast_to(np.cos(phi)[None, :, None], (nz, ny, nx)).copy()
    return lam, phi, g


def deformational_flow(nx: int, ny: int, nz: int, g: np.ndarray,
                       cmax: float = 0.6, wamp: float = 0.05,
                       scale: float = 1.0):
    """Courant fields of the 3D lat-lon case.

    Horizontal: corner stream function Psi = A sin^2(2 pi x/nx) sin^2(pi y/ny)
    (x, y corner coordinates in cells), the same on every level, scaled so the
    largest |U|/G_face or |V|/G_face is ``cmax``.  Vertical: W(k+1/2) =
    wamp * sin(lambda) * sin(2 pi (j+1/2)/ny) * sin(pi (k+1)/nz), which is 0
    on the top face.  If the outflow Courant sum exceeds 1 all three are
    scaled down together (the applied factor is returned).
    """
    xcor = np.arange(nx) + 1.0
    ycor = np.arange(ny) + 1.0
    psi_c = (np.sin(2.0 * math.pi * xcor / nx)[None, :] ** 2
             * np.sin(math.pi * ycor / ny)[:, None] ** 2)
    u2, v2 = _uv_from_corner_streamfunction(psi_c[None])
    g2 = g[0]
    gu = g2                                        # G is constant in i
    gv = 0.5 * (g2 + np.roll(g2, -1, axis=0))
    peak = max(np.max(np.abs(u2[0] / gu)), np.max(np.abs(v2[0] / gv)))
    A = cmax / peak
    u = np.broadcast_to(A * u2, (nz, ny, nx)).copy()
    v = np.broadcast_to(A * v2, (nz, ny, nx)).copy()
    lam = 2.0 * math.pi * (np.arange(nx) + 0.5) / nx
    jj = (np.arange(ny) + 0.5) / ny
    kk = np.arange(nz) + 1.0
    w = (wamp * np.sin(lam)[None, None, :] * np.sin(2.0 * math.pi * jj)[None, :, None]
         * np.sin(math.pi * kk / nz)[:, None, None])
    w[-1] = 0.0
    u *= scale
    v *= scale
    w *= scale
    s = outflow_courant_max(u, v, w, g)
    applied = 1.0
    if s > 1.0:
        applied = 0.98 / s
        u *= applied
        v *= applied
        w *= applied
    return u, v, w, applied


def latlon_3d(nx: int = 256, ny: int = 256, nz: int = 64, seed: int = DEFAULT_SEED,
              steps: int = 50, flow_scale: float = 1.0) -> Case:
    """3D lat-lon case: Gaussian blob plus a step function, deformational flow.

    Blob: amplitude 1, sigma 10 cells, centre (nx/3, ny/2, nz/2) shifted by a
    seeded sub-cell offset; step: +1 on i in [nx/2, 3nx/4), j in [ny/4, 3ny/4),
    all k; background 0.
    """
    rng = np.random.default_rng(seed)
    _, _, g = latlon_geometry(nx, ny, nz)
    u, v, w, applied = deformational_flow(nx, ny, nz, g, scale=flow_scale)
    off = rng.uniform(-0.5, 0.5, size=3)
    ci, cj, ck = nx / 3.0 + off[0], ny / 2.0 + off[1], nz / 2.0 + off[2]
    sig = 10.0
    I = np.arange(nx) + 0.5
    J = np.arange(ny) + 0.5
    K = np.arange(nz) + 0.5
    blob = (np.exp(-0.5 * ((K[:, None, None] - ck) / sig) ** 2)
            * np.exp(-0.5 * ((J[None, :, None] - cj) / sig) ** 2)
            * np.exp(-0.5 * ((I[None, None, :] - ci) / sig) ** 2))
    step = np.zeros((nz, ny, nx))
    step[:, ny // 4:(3 * ny) // 4, nx // 2:(3 * nx) // 4] = 1.0
    psi = blob + step
    return Case("latlon_3d", nx, ny, nz, psi, u, v, w, g, iord=2, nonosc=1,
                steps=steps, halo=2, meta=dict(seed=seed, flow_scale_applied=applied))


def random_case(nx: int, ny: int, nz: int, seed: int = DEFAULT_SEED,
                cmax: float = 0.2, psi_lo: float = 0.0, psi_hi: float = 1.0,
                g_lo: float = 0.5, g_hi: float = 1.5, iord: int = 2,
                nonosc: int = 1, kbc: int = 0) -> Case:
    """Unstructured random inputs (divergent flow), for parity on odd sizes.
    kbc = 1 (periodic k) keeps the top face's W; else it is the closed face."""
    rng = np.random.default_rng(seed)
    shp = (nz, ny, nx)
    psi = rng.uniform(psi_lo, psi_hi, size=shp)
    g = rng.uniform(g_lo, g_hi, size=shp)
    u = rng.uniform(-cmax, cmax, size=shp) * g
    v = rng.uniform(-cmax, cmax, size=shp) * g
    w = rng.uniform(-cmax, cmax, size=shp) * g
    if kbc != 1:
        w[-1] = 0.0
    s = outflow_courant_max(u, v, w, g, kbc)
    if s > 1.0:
        f = 0.98 / s
        u *= f
        v *= f
        w *= f
    return Case("random", nx, ny, nz, psi, u, v, w, g, iord=iord, nonosc=nonosc,
                meta=dict(seed=seed, kbc=kbc))


def nondivergent_case(nx: int, ny: int, nz: int, seed: int = DEFAULT_SEED,
                      cmax: float = 0.3, const: Optional[float] = 1.7,
                      g_lo: float = 0.5, g_hi: float = 1.5, kbc: int = 0) -> Case:
    """Random but discretely non-divergent G-weighted flow.

    Horizontal part from a random corner stream function per level; an x-z
    stream function chi at (i+1/2, j, k+1/2), zero on the bottom and top
    faces (with kbc = 1, periodic in k instead), adds U and W parts whose
    divergence also cancels exactly.  G is random and positive.  psi is the
    constant ``const`` (or random if None).
    """
    rng = np.random.default_rng(seed)
    shp = (nz, ny, nx)
    psi_c = rng.uniform(-1.0, 1.0, size=shp)
    u, v = _uv_from_corner_streamfunction(psi_c)
    chi = np.zeros((nz + 1, ny, nx))
    if kbc == 1:
        chi[1:] = rng.uniform(-1.0, 1.0, size=(nz, ny, nx))
        chi[0] = chi[nz]  # chi(-1/2) is chi(nz-1/2)
    elif nz > 1:
        chi[1:nz] = rng.uniform(-1.0, 1.0, size=(nz - 1, ny, nx))
    # U(i+1/2, j, k) -= chi(i+1/2, j, k+1/2) - chi(i+1/2, j, k-1/2)
    u = u - (chi[1:] - chi[:-1])
    # W(i, j, k+1/2) = chi(i+1/2, j, k+1/2) - chi(i-1/2, j, k+1/2)
    w = chi[1:] - np.roll(chi[1:], 1, axis=-1)
    g = rng.uniform(g_lo, g_hi, size=shp)
    s = outflow_courant_max(u, v, w, g, kbc)
    f = cmax / s
    u, v, w = u * f, v * f, w * f
    psi = np.full(shp, const) if const is not None else rng.uniform(0.5, 1.5, size=shp)
    return Case("nondivergent", nx, ny, nz, psi, u, v, w, g, meta=dict(seed=seed))


def uniform_shift_case(nx: int, ny: int, nz: int, axis: str, sign: int,
                       seed: int = DEFAULT_SEED, kbc: int = 0) -> Case:
    """Courant number exactly +-1 along one axis, 0 along the others, G = 1.

    psi is uniform in [1, 2): any two values are within a factor of two, so
    the differences the scheme forms are exact in binary floating point.
    For axis 'z' the boundary faces stay zero (W = sign inside only), unless
    kbc = 1 (periodic k: every face).
    """
    rng = np.random.default_rng(seed)
    shp = (nz, ny, nx)
    psi = rng.uniform(1.0, 2.0, size=shp)
    u = np.zeros(shp)
    v = np.zeros(shp)
    w = np.zeros(shp)
    if axis == "x":
        u[:] = float(sign)
    elif axis == "y":
        v[:] = float(sign)
    elif axis == "z":
        if kbc == 1:
            w[:] = float(sign)
        else:
            w[:-1] = float(sign)
    else:
        raise ValueError(axis)
    g = np.ones(shp)
    return Case(f"shift_{axis}{'+' if sign > 0 else '-'}", nx, ny, nz, psi, u, v, w, g,
                meta=dict(seed=seed))


def gaussian_rotation_2d(n: int, sigma_frac: float = 0.1, courant: float = 0.5,
                         background: float = 0.0):
    """Smooth Gaussian under solid-body rotation, for convergence studies.

    Rotation radius R = 0.45 n about the centre; the Gaussian (sigma =
    sigma_frac * R) starts R/2 from the centre.  omega = 2 pi / T with T the
    integer step count of one revolution at the chosen Courant number, so
    after T steps the exact solution is the initial field.
    Returns (case, T).
    """
    R = 0.45 * n
    T = int(round(2.0 * math.pi * R / courant))
    omega = 2.0 * math.pi / T
    xc = yc = n / 2.0
    xi = np.arange(n) + 1.0
    X, Y = np.meshgrid(xi, xi, indexing="xy")
    r2 = np.minimum((X - xc) ** 2 + (Y - yc) ** 2, R * R)
    psi_c = 0.5 * omega * r2
    u, v = _uv_from_corner_streamfunction(psi_c[None])
    w = np.zeros_like(u)
    g = np.ones_like(u)
    xcell = np.arange(n) + 0.5
    Xc, Yc = np.meshgrid(xcell, xcell, indexing="xy")
    sig = sigma_frac * R
    psi = background + np.exp(-0.5 * ((Xc - (xc + 0.5 * R)) ** 2 + (Yc - yc) ** 2) / sig ** 2)
    case = Case(f"gauss_rot_{n}", n, n, 1, psi[None].copy(), u, v, w, g, steps=T,
                meta=dict(omega=omega, R=R))
    return case, T


def batched_domains(ndomains: int = 64, ntracers: int = 8, seed: int = DEFAULT_SEED,
                    lo=(32, 32, 16), hi=(256, 256, 64)) -> List[Case]:
    """Independent domains with log-uniform sizes, each carrying ``ntracers``.

    nx, ny ~ logU[lo, hi] and nz ~ logU[lo_z, hi_z], drawn independently and
    rounded to integers.  Each domain gets the lat-lon deformational flow of
    its own size; its tracers are uniform[0, 1) plus one Gaussian blob of
    random centre and width.
    """
    rng = np.random.default_rng(seed)
    out = []
    for d in range(ndomains):
        dims = [int(round(math.exp(rng.uniform(math.log(lo[a]), math.log(hi[a])))))
                for a in range(3)]
        nx, ny, nz = dims
        _, _, g = latlon_geometry(nx, ny, nz)
        u, v, w, _ = deformational_flow(nx, ny, nz, g)
        psi = np.empty((ntracers, nz, ny, nx))
        I = np.arange(nx) + 0.5
        J = np.arange(ny) + 0.5
        K = np.arange(nz) + 0.5
        for t in range(ntracers):
            base = rng.uniform(0.0, 1.0, size=(nz, ny, nx))
            c = rng.uniform(0.2, 0.8, size=3) * np.array([nz, ny, nx])
            sg = rng.uniform(0.05, 0.2) * min(nx, ny)
            blob = (np.exp(-0.5 * ((K[:, None, None] - c[0]) / max(sg, 2.0)) ** 2)
                    * np.exp(-0.5 * ((J[None, :, None] - c[1]) / sg) ** 2)
                    * np.exp(-0.5 * ((I[None, None, :] - c[2]) / sg) ** 2))
            psi[t] = base + blob
        out.append(Case(f"domain{d}", nx, ny, nz, psi, u, v, w, g, iord=2, nonosc=1,
                        meta=dict(seed=seed, index=d)))
    return out
