"""Seeded synthetic inputs for the Poisson solvers.

This module only produces input data: node coordinates, densities, boundary
potentials of textbook closed forms and request streams.  It holds none of the
solver arithmetic, so both the CUDA path and the FP64 CPU oracle may use it.

Conventions (shared by every consumer):

* Cartesian "N^3" means N intervals per axis on [lo, hi]^3, nodes 0..N,
  (N-1)^3 interior unknowns (vertex-centred grids, Sec. 2.1.3).  A field is a
  C-ordered array of shape (nz+2g-1, ny+2g-1, nx+2g-1), x fastest, where g is
  the stencil radius (1 for the 7-point, 2 for the 13-point Laplacian); node
  index i sits at array index i+g-1.
* Spherical grids (Eq. 2) store (Nphi+2, Ntheta+2, Nr+2) with r fastest; node
  (i, j, k) sits at array index (k+1, j+1, i+1); the ghost layers hold the
  inner mirror, the pole slots, the periodic copies and the outer boundary.
* Random numbers come from numpy's PCG64 with fixed seeds.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "cart_shape", "cart_coords", "uniform_sphere", "gaussian_blobs",
    "gaussian_blob_params", "gaussian_blobs_device", "lognormal_field", "lognormal_field_device",
    "manufactured_sine",
    "smooth_sphere_density", "spherical_coords", "spherical_density",
    "ServingRequest", "serving_stream", "rng",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def cart_shape(n, order: int):
    """Array shape (z, y, x) of a Cartesian field with n=(nx,ny,nz) intervals."""
    g = order // 2
    nx, ny, nz = (n, n, n) if np.isscalar(n) else n
    return (nz + 2 * g - 1, ny + 2 * g - 1, nx + 2 * g - 1)


def cart_coords(n, order: int, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    """Node coordinates (x, y, z) as 1-D arrays covering the whole array,
    ghost layers included."""
    g = order // 2
    nn = (n, n, n) if np.isscalar(n) else tuple(n)
    out = []
    for a in range(3):
        h = (hi[a] - lo[a]) / nn[a]
        idx = np.arange(-(g - 1), nn[a] + g, dtype=np.float64)
        out.append(lo[a] + idx * h)
    return tuple(out)


def _mesh(n, order, lo, hi):
    x, y, z = cart_coords(n, order, lo, hi)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def uniform_sphere(n: int, order: int = 2, radius: float = 0.25, rho0: float = 1.0,
                   G: float = 1.0, centre=(0.5, 0.5, 0.5)):
    """Uniform sphere of density rho0 in the unit box.

    Returns (rho, phi0, phi_exact): phi0 is zero on interior nodes and carries
    the closed-form potential on the boundary (and ghost) nodes, so it serves
    both as a cold-start guess and as Dirichlet data.  The closed form is the
    textbook potential of a uniform ball: 2 pi G rho0 (r^2/3 - a^2) inside,
    -G M / r outside, M = 4 pi rho0 a^3 / 3.
    """
    X, Y, Z = _mesh(n, order, (0, 0, 0), (1, 1, 1))
    r = np.sqrt((X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2)
    rho = np.where(r < radius, rho0, 0.0)
    mass = 4.0 * math.pi * rho0 * radius ** 3 / 3.0
    with np.errstate(divide="ignore"):
        outside = -G * mass / np.maximum(r, 1e-300)
    phi_exact = np.where(r < radius, 2.0 * math.pi * G * rho0 * (r * r / 3.0 - radius ** 2), outside)
    phi0 = phi_exact.copy()
    g = order // 2
    phi0[g:-g, g:-g, g:-g] = 0.0
    return rho, phi0, phi_exact


@dataclass
class Blob:
    centre: tuple
    sigma: float
    amp: float


def gaussian_blob_params(seed: int, nblobs: int = 8):
    """Blob parameters drawn per blob in the order centre (3), sigma, amplitude:
    centres U[0.2,0.8]^3, sigma U[0.02,0.08], amplitude U[0.5,2]."""
    g = rng(seed)
    blobs = []
    for _ in range(nblobs):
        c = tuple(g.uniform(0.2, 0.8, size=3))
        s = float(g.uniform(0.02, 0.08))
        a = float(g.uniform(0.5, 2.0))
        blobs.append(Blob(c, s, a))
    return blobs


def gaussian_blobs(n: int, order: int = 2, seed: int = 2, nblobs: int = 8, blobs=None,
                   shift=(0.0, 0.0, 0.0)):
    """Sum of isotropic Gaussians A exp(-|x-c|^2/(2 sigma^2)) sampled on the
    nodes of the unit box; `shift` translates every centre."""
    if blobs is None:
        blobs = gaussian_blob_params(seed, nblobs)
    x, y, z = cart_coords(n, order)
    rho = np.zeros((z.size, y.size, x.size))
    for b in blobs:
        cx, cy, cz = (b.centre[a] + shift[a] for a in range(3))
        w = -0.5 / (b.sigma * b.sigma)
        ex = np.exp(w * (x - cx) ** 2)
        ey = np.exp(w * (y - cy) ** 2)
        ez = np.exp(w * (z - cz) ** 2)
        rho += b.amp * ez[:, None, None] * ey[None, :, None] * ex[None, None, :]
    return rho


def gaussian_blobs_device(n: int, blobs, device, order: int = 2, shift=(0.0, 0.0, 0.0)):
    """gaussian_blobs() evaluated with torch on `device` (same separable
    formula, float64), for request streams whose densities are made on the GPU."""
    import torch
    g = order // 2
    idx = torch.arange(-(g - 1), n + g, dtype=torch.float64, device=device)
    x = idx * (1.0 / n)
    rho = torch.zeros((x.numel(),) * 3, dtype=torch.float64, device=device)
    for b in blobs:
        cx, cy, cz = (b.centre[a] + shift[a] for a in range(3))
        w = -0.5 / (b.sigma * b.sigma)
        ex = torch.exp(w * (x - cx) ** 2)
        ey = torch.exp(w * (x - cy) ** 2)
        ez = torch.exp(w * (x - cz) ** 2)
        rho += b.amp * ez[:, None, None] * ey[None, :, None] * ex[None, None, :]
    return rho


def lognormal_field(n: int, order: int = 4, seed: int = 3, slope: float = -11.0 / 3.0):
    """Lognormal turbulent-like density: a Gaussian random field g with 3-D
    power spectrum P(k) ~ |k|^slope (k=0 zeroed) on the periodic N^3 lattice,
    standardised to unit variance, then rho = exp(g - 1/2) so that
    sigma(ln rho) = 1 and <rho> ~ 1.  Node N repeats node 0."""
    g = rng(seed)
    white = g.standard_normal((n, n, n))
    wk = np.fft.rfftn(white)
    kz = np.fft.fftfreq(n)[:, None, None]
    ky = np.fft.fftfreq(n)[None, :, None]
    kx = np.fft.rfftfreq(n)[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    amp = k2 ** (slope / 4.0)          # sqrt(P(k)) with P ~ k^slope
    amp[0, 0, 0] = 0.0
    field_ = np.fft.irfftn(wk * amp, s=(n, n, n))
    field_ -= field_.mean()
    field_ /= field_.std()
    rho_p = np.exp(field_ - 0.5)
    gh = order // 2
    idx = (np.arange(-(gh - 1), n + gh) % n)
    return rho_p[np.ix_(idx, idx, idx)]


def lognormal_field_device(n: int, device, order: int = 4, seed: int = 3,
                           slope: float = -11.0 / 3.0):
    """lognormal_field() with the FFT done by torch on `device` (same seeded
    white noise from PCG64, same spectrum and standardisation), for grids where
    a host FFT would take minutes."""
    import torch
    g = rng(seed)
    white = torch.from_numpy(g.standard_normal((n, n, n))).to(device)
    wk = torch.fft.rfftn(white)
    del white
    fz = torch.fft.fftfreq(n, device=device, dtype=torch.float64)
    fx = torch.fft.rfftfreq(n, device=device, dtype=torch.float64)
    k2 = fx[None, None, :] ** 2 + fz[None, :, None] ** 2 + fz[:, None, None] ** 2
    k2[0, 0, 0] = 1.0
    amp = k2 ** (slope / 4.0)
    amp[0, 0, 0] = 0.0
    wk *= amp
    del amp, k2
    field_ = torch.fft.irfftn(wk, s=(n, n, n))
    del wk
    field_ -= field_.mean()
    field_ /= field_.std(unbiased=False)
    rho_p = torch.exp(field_ - 0.5)
    del field_
    gh = order // 2
    idx = torch.arange(-(gh - 1), n + gh, device=device) % n
    return rho_p[idx][:, idx][:, :, idx].contiguous()


def manufactured_sine(n: int, order: int, G: float = 1.0):
    """Phi = sin(pi x) sin(pi y) sin(pi z) on [0,1]^3 with its density
    rho = -3 pi^2 Phi / (4 pi G).  Returns (rho, phi0, phi_exact); phi0 has the
    exact values on boundary and ghost nodes and zero inside."""
    X, Y, Z = _mesh(n, order, (0, 0, 0), (1, 1, 1))
    phi = np.sin(math.pi * X) * np.sin(math.pi * Y) * np.sin(math.pi * Z)
    rho = -3.0 * math.pi ** 2 * phi / (4.0 * math.pi * G)
    phi0 = phi.copy()
    g = order // 2
    phi0[g:-g, g:-g, g:-g] = 0.0
    return rho, phi0, phi


def smooth_sphere_density(n, order, centres, radii, masses, lo=(-1, -1, -1), hi=(1, 1, 1)):
    """The (1-w^2)^2 spheres of Sec. 3.1: rho_p (1 - (d/a_p)^2)^2 inside d < a_p,
    rho_p = M_p / (32 pi a_p^3 / 105)."""
    X, Y, Z = _mesh(n, order, lo, hi)
    rho = np.zeros_like(X)
    for c, a, m in zip(centres, radii, masses):
        rp = m / (32.0 * math.pi * a ** 3 / 105.0)
        d = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
        w2 = (d / a) ** 2
        rho += np.where(d < a, rp * (1.0 - w2) ** 2, 0.0)
    return rho


def spherical_coords(nr: int = 256, nth: int = 128, nph: int = 256, r_in: float = 0.01,
                     r_out: float = 1.0):
    """Node coordinates of the spherical grid: r log-spaced from r_in to r_out
    (nr nodes), theta_j = (j+1/2) pi / nth, phi_k = 2 pi k / nph."""
    i = np.arange(nr, dtype=np.float64)
    r = r_in * (r_out / r_in) ** (i / (nr - 1))
    r[0], r[-1] = r_in, r_out
    th = (np.arange(nth) + 0.5) * math.pi / nth
    ph = 2.0 * math.pi * np.arange(nph) / nph
    return r, th, ph


def spherical_density(r, th, ph, with_angles: bool = True):
    """rho = r^-2 (1 + 0.1 cos 2 phi)(1 + 0.2 cos^2 theta) on the node grid,
    returned in the (Nphi+2, Ntheta+2, Nr+2) ghosted layout (ghosts zero)."""
    rho = np.zeros((ph.size + 2, th.size + 2, r.size + 2))
    fr = r ** -2.0
    if with_angles:
        fth = 1.0 + 0.2 * np.cos(th) ** 2
        fph = 1.0 + 0.1 * np.cos(2.0 * ph)
    else:
        fth = np.ones_like(th)
        fph = np.ones_like(ph)
    rho[1:-1, 1:-1, 1:-1] = fph[:, None, None] * fth[None, :, None] * fr[None, None, :]
    return rho


@dataclass
class ServingRequest:
    rid: int
    arrival_s: float
    n: int
    tol: float
    blobs: list
    seq_id: int = -1          # >= 0: member of a warm-started sequence
    seq_step: int = 0
    shift: tuple = field(default=(0.0, 0.0, 0.0))


def serving_stream(n_requests: int = 2000, rate_hz: float = 200.0, seed: int = 5,
                   sizes=(32, 64, 96, 128, 192, 256), seq_fraction: float = 0.3,
                   seq_len: int = 10, step_shift: float = 0.01):
    """Request stream: Poisson arrivals (exponential gaps of mean 1/rate),
    cube sizes uniform over `sizes`, 1-16 Gaussian blobs, tolerance 1e-6 or
    1e-10 with probability 1/2.  A fraction `seq_fraction` of the requests
    belongs to sequences of `seq_len` steps whose blobs translate by
    `step_shift` per step along a fixed seeded direction."""
    g = rng(seed)
    gaps = g.exponential(1.0 / rate_hz, size=n_requests)
    t = np.cumsum(gaps)
    n_seq_req = int(round(seq_fraction * n_requests)) // seq_len * seq_len
    n_seq = n_seq_req // seq_len
    # sequence members are interleaved through the stream at seeded slots
    slots = np.sort(g.choice(n_requests, size=n_seq_req, replace=False))
    seq_of_slot = np.repeat(np.arange(n_seq), seq_len)
    g.shuffle(seq_of_slot)
    seq_params = []
    for s in range(n_seq):
        nsz = int(g.choice(sizes))
        nb = int(g.integers(1, 17))
        blobs = [Blob(tuple(g.uniform(0.3, 0.7, size=3)), float(g.uniform(0.02, 0.08)),
                      float(g.uniform(0.5, 2.0))) for _ in range(nb)]
        d = g.standard_normal(3)
        d /= np.linalg.norm(d)
        tol = 1e-6 if g.uniform() < 0.5 else 1e-10
        seq_params.append((nsz, blobs, tuple(d), tol))
    slot_to_seq = dict(zip(slots.tolist(), seq_of_slot.tolist()))
    step_count = [0] * n_seq
    out = []
    for rid in range(n_requests):
        if rid in slot_to_seq:
            s = slot_to_seq[rid]
            nsz, blobs, d, tol = seq_params[s]
            k = step_count[s]
            step_count[s] += 1
            shift = tuple(step_shift * k * d[a] for a in range(3))
            out.append(ServingRequest(rid, float(t[rid]), nsz, tol, blobs, s, k, shift))
        else:
            nsz = int(g.choice(sizes))
            nb = int(g.integers(1, 17))
            blobs = [Blob(tuple(g.uniform(0.2, 0.8, size=3)), float(g.uniform(0.02, 0.08)),
                          float(g.uniform(0.5, 2.0))) for _ in range(nb)]
            tol = 1e-6 if g.uniform() < 0.5 else 1e-10
            out.append(ServingRequest(rid, float(t[rid]), nsz, tol, blobs))
    return out


# ------------------------------------------------------------------ zero-padded radial grid
# Sec. 2.2 / Sec. 3.3: the multipole expansions are more accurate when no mass
# lies near the radii where they are evaluated, so the grid of the potential is
# extended inward and outward beyond the active range r_in < r < r_out, the
# density is zero in the extensions, and the expansions are written at the
# extended ends (the ghost shells next to the first and last nodes).  The
# active range is logarithmic; the outer extension continues it; the inner
# extension (where continuing the logarithmic grid would make the spacing
# needlessly small) continues it smoothly with a fourth-order polynomial in the
# node index that matches the logarithmic grid's value, first and second
# derivative at r_in and reaches r_in_pad with a chosen end spacing.  These are
# node coordinates handed to poisson_create, i.e. an input of the solve.

def padded_log_radii(r_in: float, r_out: float, n: int, n_pad_in: int = 20, n_pad_out: int = 20,
                     r_in_pad: float | None = None, end_spacing: float | None = None):
    """Node radii of a logarithmic grid of n nodes on [r_in, r_out] with n_pad_in
    inner and n_pad_out outer extension nodes.  Returns (r, active) where
    `active` is the boolean mask of the n logarithmic nodes (the density must be
    zero elsewhere).  r_in_pad defaults to r_in / 2; end_spacing (the node
    spacing at r_in_pad) defaults to the mean spacing of the inner extension."""
    if not (0.0 < r_in < r_out) or n < 3:
        raise ValueError("need 0 < r_in < r_out and n >= 3")
    q = (r_out / r_in) ** (1.0 / (n - 1))
    lq = math.log(q)
    i = np.arange(n, dtype=np.float64)
    core = r_in * q ** i
    core[0], core[-1] = r_in, r_out
    out = r_out * q ** np.arange(1, n_pad_out + 1, dtype=np.float64)
    inner = np.zeros(0)
    if n_pad_in > 0:
        rp = r_in / 2.0 if r_in_pad is None else float(r_in_pad)
        if not (0.0 < rp < r_in):
            raise ValueError("need 0 < r_in_pad < r_in")
        m = n_pad_in
        ds = (r_in - rp) / m if end_spacing is None else float(end_spacing)
        # r(s) = r_in + a1 s + a2 s^2 + a3 s^3 + a4 s^4 for s in [-m, 0]:
        # C2 join with r_in q^s at s = 0, r(-m) = rp, r'(-m) = ds
        a1, a2 = r_in * lq, r_in * lq * lq / 2.0
        A = np.array([[-m ** 3, m ** 4], [3.0 * m * m, -4.0 * m ** 3]])
        rhs = np.array([rp - r_in + a1 * m - a2 * m * m, ds - a1 + 2.0 * a2 * m])
        a3, a4 = np.linalg.solve(A, rhs)
        s = -np.arange(m, 0, -1, dtype=np.float64)
        inner = r_in + a1 * s + a2 * s * s + a3 * s ** 3 + a4 * s ** 4
        if not np.all(np.diff(np.concatenate([inner, [r_in]])) > 0.0):
            raise ValueError("the inner extension is not monotone; adjust n_pad_in, r_in_pad or end_spacing")
    r = np.concatenate([inner, core, out])
    active = np.zeros(r.size, dtype=bool)
    active[inner.size:inner.size + n] = True
    return r, active
