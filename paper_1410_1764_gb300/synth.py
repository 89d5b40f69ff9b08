"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

This module holds only input recipes (initial data, patch sizes, wave-speed
fields, receiver positions): none of the method's arithmetic.  Every array is
float64, padded with ghost zones of width g that are left at zero (callers
fill them), shaped (nvars, nz+2g, ny+2g, nx+2g) with x fastest.

Grid convention: periodic, N points per axis at x_i = i h, h = L / N, L = 1.
"""
import numpy as np

L_BOX = 1.0

# BSSN variable order and the flat-space value of each variable
BSSN_NAMES = (["phi", "gt_xx", "gt_xy", "gt_xz", "gt_yy", "gt_yz", "gt_zz", "K",
               "At_xx", "At_xy", "At_xz", "At_yy", "At_yz", "At_zz",
               "Xt_x", "Xt_y", "Xt_z", "alpha", "beta_x", "beta_y", "beta_z",
               "B_x", "B_y", "B_z"])
BSSN_FLAT = np.array([0.0, 1, 0, 0, 1, 0, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0])


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def pad(interior, g):
    """Embed (nv, nz, ny, nx) interior data in a zero-ghost padded array."""
    interior = np.asarray(interior, dtype=np.float64)
    if interior.ndim == 3:
        interior = interior[None]
    nv, nz, ny, nx = interior.shape
    out = np.zeros((nv, nz + 2 * g, ny + 2 * g, nx + 2 * g))
    out[:, g:g + nz, g:g + ny, g:g + nx] = interior
    return out


def interior(a, g):
    return a[..., g:a.shape[-3] - g, g:a.shape[-2] - g, g:a.shape[-1] - g]


def coords(nx, ny, nz, L=L_BOX):
    """Vertex coordinates x_i = i L/N (index order z, y, x)."""
    h = L / nx
    x = np.arange(nx) * (L / nx)
    y = np.arange(ny) * (L / ny)
    z = np.arange(nz) * (L / nz)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z, h


def plane_wave(n, g, L=L_BOX):
    """Wave 32^3 recipe: u = sin(k.x), k = 2pi/L (1,1,1), travelling along +k,
    rho = du/dt of the continuum solution sin(k.x - w t), w = |k|."""
    X, Y, Z, h = coords(n, n, n, L)
    k = 2 * np.pi / L
    w = k * np.sqrt(3.0)
    ph = k * (X + Y + Z)
    return pad(np.stack([np.sin(ph), -w * np.cos(ph)]), g), h


def gaussian_pulses(n, g, seed, npulse=8, width=0.05, L=L_BOX):
    """Wave 256^3 recipe: u = sum_k A_k exp(-r_k^2 / (2 W^2)), W = 0.05 L,
    centres uniform in the box, A_k ~ N(0,1), r_k the periodic minimum-image
    distance; rho = 0.  Draw order: centres (npulse x 3), then amplitudes."""
    r = rng(seed)
    centres = r.uniform(0.0, L, size=(npulse, 3))
    amps = r.standard_normal(npulse)
    X, Y, Z, h = coords(n, n, n, L)
    u = np.zeros_like(X)
    W = width * L
    for c, A in zip(centres, amps):
        d2 = np.zeros_like(X)
        for Q, q in ((X, c[0]), (Y, c[1]), (Z, c[2])):
            dq = Q - q
            dq -= L * np.round(dq / L)
            d2 += dq * dq
        u += A * np.exp(-0.5 * d2 / (W * W))
    return pad(np.stack([u, np.zeros_like(u)]), g), h


def bssn_noise(nx, ny, nz, g, seed, amp=1e-10, r=None):
    """BSSN flat space plus independent uniform noise U(-amp, amp) on each of
    the 24 variables at each point.  h = L / nx."""
    r = r if r is not None else rng(seed)
    noise = r.uniform(-amp, amp, size=(24, nz, ny, nx))
    data = BSSN_FLAT[:, None, None, None] + noise
    return pad(data, g), L_BOX / nx


def patch_dims(seed, npatch=64, lo=16, hi=96):
    """Batched-patch recipe: each side an integer uniform in [lo, hi]."""
    return rng(seed).integers(lo, hi + 1, size=(npatch, 3))


def bssn_patches(seed, npatch=64, g=3, amp=1e-10, lo=16, hi=96, h=1.0 / 64):
    """Patch states (list of padded arrays, dims (nx, ny, nz)) and their h.
    All patches share h (one refinement level); sizes first, then noise."""
    r = rng(seed)
    dims = r.integers(lo, hi + 1, size=(npatch, 3))
    states = []
    for nx, ny, nz in dims:
        st, _ = bssn_noise(int(nx), int(ny), int(nz), g, None, amp, r=r)
        states.append(st)
    return states, dims, h


def smooth_field(n, seed, sigma_cells=4.0):
    """White N(0,1) noise on an n^3 grid, periodic Gaussian filter of width
    sigma_cells (FFT), scaled to max |F| = 1."""
    F = rng(seed).standard_normal((n, n, n))
    k = np.fft.fftfreq(n) * 2 * np.pi
    KZ, KY, KX = np.meshgrid(k, k, k, indexing="ij")
    filt = np.exp(-0.5 * sigma_cells ** 2 * (KX ** 2 + KY ** 2 + KZ ** 2))
    F = np.real(np.fft.ifftn(np.fft.fftn(F) * filt))
    return F / np.max(np.abs(F))


def wave_speed(n, g, seed, amp=0.2):
    """Adjoint recipe: c = 1 + amp F with F a smooth periodic random field."""
    return pad(1.0 + amp * smooth_field(n, seed), g)[0]


def receivers(n, g, seed, nrecv=512):
    """nrecv distinct interior points, as padded linear indices into one
    grid function of an n^3 grid with ghost width g."""
    flat = rng(seed).choice(n * n * n, size=nrecv, replace=False)
    k, rem = np.divmod(flat, n * n)
    j, i = np.divmod(rem, n)
    p = n + 2 * g
    return ((k + g) * p + (j + g)) * p + (i + g)


def adjoint_problem(n=128, g=2, seed=4, npulse=8, nrecv=512):
    """Initial state (Gaussian pulses, rho = 0), trial speed c, receiver
    indices and the seed of the 'true' speed used to synthesise data."""
    y0, h = gaussian_pulses(n, g, seed, npulse=npulse)
    c = wave_speed(n, g, seed)
    recv = receivers(n, g, seed, nrecv)
    return y0, c, recv, h, seed + 1


def amr_boxes(seed, nc=128, lo=8, hi=24, margin_lo=5, margin_hi=6):
    """Mesh-refinement recipe: 8 boxes, one per octant of an nc^3 coarse
    grid, each side an integer uniform in [lo, hi] coarse points, placed
    uniformly inside its octant and at least margin_lo / margin_hi points
    from the grid's faces (so boxes are disjoint and their prolongation
    stays on the grid).  Returns a list of (lo, hi) per box, x fastest."""
    r = rng(seed)
    half = nc // 2
    boxes = []
    for o in range(8):
        oc = (o & 1, (o >> 1) & 1, (o >> 2) & 1)
        side = r.integers(lo, hi + 1, size=3)
        blo, bhi = [], []
        for d in range(3):
            a = max(margin_lo, oc[d] * half)
            b = min((oc[d] + 1) * half, nc - margin_hi) - int(side[d])
            x = int(r.integers(a, b + 1))
            blo.append(x)
            bhi.append(x + int(side[d]))
        boxes.append((tuple(blo), tuple(bhi)))
    return boxes
