"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws and shapes inputs: velocity models, acquisition geometry,
frequencies and right-hand sides.  It holds none of the method's arithmetic (no
assembly, no solve, no derivative), so both the CUDA path and the CPU oracle may
use it without sharing any of the computation they are compared on.

Geometry conventions (all workloads): the domain is [0, lx] x [0, lz] with z = 0
the top (surface) row; the grid has nx x nz nodes, node (i, j) sits at
(x, z) = (i*hx, j*hz) with hx = lx/(nx-1), hz = lz/(nz-1), and the canonical
node index is k = i*nz + j (z fastest, the Kronecker order of the regulariser
D_x = D_nx (x) I_nz of Section 2, Eq. (ThisGamma)).

The paper's experiments use the smoothed Marmousi model (Section 4), which is not
available here; the velocity generators below are seeded stand-ins with the same
character: smooth, layered, wavespeed increasing with depth, speeds 1.5-4.5.
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "Acquisition", "Workload", "gaussian_inclusion_velocity", "gaussian_random_field",
    "layered_velocity", "gaussian_smooth", "top_row_sources", "surface_receivers",
    "config_plain", "config_fwi_step", "config_mixed", "config_hypergrad", "tiny_case",
    "random_rhs", "resample_bilinear", "sample_on_grid",
]


@dataclasses.dataclass
class Acquisition:
    """Source and receiver positions in physical coordinates (x, z)."""
    src_xz: np.ndarray            # [n_src, 2] float64
    rec_xz: np.ndarray            # [n_rec, 2] float64
    src_amp: np.ndarray | None = None   # [n_src] float64, default 1
    rec_w: np.ndarray | None = None     # [n_rec] float64 receiver weights, default 1

    @property
    def n_src(self) -> int:
        return int(self.src_xz.shape[0])

    @property
    def n_rec(self) -> int:
        return int(self.rec_xz.shape[0])


@dataclasses.dataclass
class Workload:
    """One named synthetic workload (grid, models, frequencies, acquisition)."""
    name: str
    nx: int
    nz: int
    lx: float
    lz: float
    omegas: np.ndarray            # [n_omega] angular frequencies
    m: np.ndarray                 # [nx*nz] squared slowness of the model being solved on
    acq: Acquisition
    m_true: np.ndarray | None = None   # [nx*nz] training model m' (data come from it)
    alpha: float = 1e-3
    mu: float = 1e-6
    extra: dict = dataclasses.field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return self.nx * self.nz

    def describe(self) -> dict:
        return {"workload": self.name, "grid": [self.nx, self.nz], "n_omega": int(len(self.omegas)),
                "n_src": self.acq.n_src, "n_rec": self.acq.n_rec}


# ----------------------------------------------------------------------------- grids

def _coords(nx: int, nz: int, lx: float, lz: float):
    x = np.linspace(0.0, lx, nx)
    z = np.linspace(0.0, lz, nz)
    X, Z = np.meshgrid(x, z, indexing="ij")     # [nx, nz], node (i, j)
    return X, Z


def _flat(field2d: np.ndarray) -> np.ndarray:
    """[nx, nz] -> canonical vector with k = i*nz + j."""
    return np.ascontiguousarray(field2d, dtype=np.float64).reshape(-1)


def sample_on_grid(fn, nx, nz, lx=1.0, lz=1.0) -> np.ndarray:
    """fn(X, Z) evaluated at the nodes of an nx x nz grid (flat, canonical order)."""
    X, Z = _coords(nx, nz, lx, lz)
    return _flat(fn(X, Z))


def resample_bilinear(field: np.ndarray, nx: int, nz: int, nx2: int, nz2: int) -> np.ndarray:
    """A nodal field on an nx x nz grid, interpolated bilinearly to the nodes of an nx2 x nz2
    grid of the same domain (flat, canonical order).  Used to carry a model between the grid
    the data are generated on and the grid it is reconstructed on."""
    f = np.asarray(field, dtype=np.float64).reshape(nx, nz)
    tx = np.linspace(0.0, nx - 1, nx2)
    tz = np.linspace(0.0, nz - 1, nz2)
    i0 = np.minimum(np.floor(tx).astype(np.int64), nx - 2)
    j0 = np.minimum(np.floor(tz).astype(np.int64), nz - 2)
    fx = (tx - i0)[:, None]
    fz = (tz - j0)[None, :]
    I, J = i0[:, None], j0[None, :]
    out = ((1 - fx) * (1 - fz) * f[I, J] + fx * (1 - fz) * f[I + 1, J]
           + (1 - fx) * fz * f[I, J + 1] + fx * fz * f[I + 1, J + 1])
    return _flat(out)


# ------------------------------------------------------------------- velocity models

def gaussian_inclusion_velocity(nx, nz, lx=1.0, lz=1.0, c0=1.0, dc=0.2, centre=(0.5, 0.6), radius=0.15):
    """c = c0 + dc * exp(-|x - centre|^2 / radius^2); returns m = 1/c^2 (flat)."""
    X, Z = _coords(nx, nz, lx, lz)
    r2 = (X - centre[0]) ** 2 + (Z - centre[1]) ** 2
    c = c0 + dc * np.exp(-r2 / radius ** 2)
    return _flat(1.0 / c ** 2)


def gaussian_random_field(nx, nz, corr_len, seed, lx=1.0, lz=1.0):
    """White noise (PCG64, seed) filtered to a Gaussian covariance exp(-r^2/(2 l^2)).

    Returns a zero-mean field [nx, nz] normalised to max |g| = 1.  The filter is
    applied with periodic FFT on a padded grid so that the edges are not wrapped.
    """
    rng = np.random.default_rng(seed)
    hx, hz = lx / (nx - 1), lz / (nz - 1)
    px = nx + int(np.ceil(4 * corr_len / hx))
    pz = nz + int(np.ceil(4 * corr_len / hz))
    w = rng.standard_normal((px, pz))
    kx = 2 * np.pi * np.fft.fftfreq(px, d=hx)
    kz = 2 * np.pi * np.fft.fftfreq(pz, d=hz)
    KX, KZ = np.meshgrid(kx, kz, indexing="ij")
    amp = np.exp(-0.25 * corr_len ** 2 * (KX ** 2 + KZ ** 2))   # sqrt of Gaussian spectrum
    g = np.real(np.fft.ifft2(np.fft.fft2(w) * amp))[:nx, :nz]
    g = g - g.mean()
    return g / np.abs(g).max()


def gaussian_smooth(field2d: np.ndarray, sigma_nodes: float) -> np.ndarray:
    """Separable Gaussian smoothing (reflecting edges), sigma in grid nodes."""
    if sigma_nodes <= 0:
        return field2d.copy()
    rad = int(np.ceil(4 * sigma_nodes))
    t = np.arange(-rad, rad + 1)
    k = np.exp(-0.5 * (t / sigma_nodes) ** 2)
    k /= k.sum()
    out = field2d
    for axis in (0, 1):
        pad = [(0, 0), (0, 0)]
        pad[axis] = (rad, rad)
        f = np.pad(out, pad, mode="reflect")
        out = np.apply_along_axis(lambda v: np.convolve(v, k, mode="valid"), axis, f)
    return out


def layered_velocity(nx, nz, seed, lx=1.0, lz=1.0, vmin=1.5, vmax=4.5):
    """Layered model: 4-6 undulating interfaces, speeds increasing with depth from
    vmin to vmax, one +-15 % Gaussian inclusion (sigma 0.08), smoothed with
    sigma = 2h.  Returns m = 1/c^2 (flat)."""
    rng = np.random.default_rng(seed)
    X, Z = _coords(nx, nz, lx, lz)
    n_if = int(rng.integers(4, 7))
    depths = np.sort(rng.uniform(0.12, 0.9, n_if)) * lz
    speeds = np.linspace(vmin, vmax, n_if + 1)
    c = np.full_like(X, speeds[0])
    for q, d0 in enumerate(depths):
        tilt = rng.uniform(-0.15, 0.15)
        amp = rng.uniform(0.0, 0.04) * lz
        wav = rng.uniform(1.0, 3.0)
        ph = rng.uniform(0, 2 * np.pi)
        surf = d0 + tilt * (X - 0.5 * lx) + amp * np.sin(2 * np.pi * wav * X / lx + ph)
        c = np.where(Z >= surf, speeds[q + 1], c)
    cx, cz = rng.uniform(0.25, 0.75) * lx, rng.uniform(0.3, 0.8) * lz
    sign = rng.choice([-1.0, 1.0])
    c = c * (1.0 + sign * 0.15 * np.exp(-((X - cx) ** 2 + (Z - cz) ** 2) / (2 * 0.08 ** 2)))
    c = gaussian_smooth(c, 2.0)
    return _flat(1.0 / c ** 2)


# ------------------------------------------------------------------------ acquisition

def top_row_sources(nx, n_src, lx=1.0):
    """n_src sources on top-row nodes i = round((q + 1/2) (nx - 1) / n_src)."""
    hx = lx / (nx - 1)
    idx = np.round((np.arange(n_src) + 0.5) * (nx - 1) / n_src).astype(np.int64)
    return np.stack([idx * hx, np.zeros(n_src)], axis=1)


def surface_receivers(n_rec, lx=1.0, z=0.0):
    """n_rec receivers at x = (r + 1/2) lx / n_rec on the line z (off-grid in x)."""
    x = (np.arange(n_rec) + 0.5) * lx / n_rec
    return np.stack([x, np.full(n_rec, z)], axis=1)


def random_rhs(n_nodes, n_rhs, seed, n_omega=1):
    """[n_omega, n_rhs, n_nodes] complex128 with N(0,1) real and imaginary parts."""
    rng = np.random.default_rng(seed)
    shape = (n_omega, n_rhs, n_nodes)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ---------------------------------------------------------------------------- configs

def config_plain(n=64):
    """Plain forward solve: unit square, n x n nodes, omega = 10, c = 1 with a Gaussian
    inclusion 1.2 (radius 0.15) at (x, z) = (0.5, 0.6), 8 top-row sources, 16 surface
    receivers."""
    m = gaussian_inclusion_velocity(n, n)
    acq = Acquisition(top_row_sources(n, 8), surface_receivers(16))
    return Workload("plain_forward_64", n, n, 1.0, 1.0, np.array([10.0]), m, acq)


def config_fwi_step(n=128, seed=2):
    """FWI step: n x n, c' = 1 + 0.3 g (g a Gaussian random field, correlation length
    0.1, seed 2), start/current model c = 1, omega in {5, 10, 15}, 16 sources, 32
    receivers, alpha = 1e-3, mu = 1e-6."""
    g = gaussian_random_field(n, n, 0.1, seed)
    m_true = _flat(1.0 / (1.0 + 0.3 * g) ** 2)
    m = np.ones(n * n)
    acq = Acquisition(top_row_sources(n, 16), surface_receivers(32))
    return Workload("fwi_step_128", n, n, 1.0, 1.0, np.array([5.0, 10.0, 15.0]), m, acq,
                    m_true=m_true, alpha=1e-3, mu=1e-6)


def config_hyper_step(n=128, seed=2):
    """Hypergradient pass on the FWI-step geometry: the training model m' is the FWI-step
    ground truth and the lower-level reconstruction is stood in for by m' smoothed with
    sigma = 4h (the hypergradient is evaluated at a given m)."""
    w = config_fwi_step(n, seed)
    m_fwi = _flat(gaussian_smooth(w.m_true.reshape(n, n), 4.0))
    w.name = f"hypergrad_step_{n}"
    w.m = m_fwi
    return w


def config_mixed(n=256, seed=3):
    """Mixed precision: n x n, omega in {5, 10, ..., 40}, c = 1 + 2 (g - min)/(max - min)
    (Gaussian random field, correlation length 0.1, seed 3), 64 top-row sources."""
    g = gaussian_random_field(n, n, 0.1, seed)
    c = 1.0 + 2.0 * (g - g.min()) / (g.max() - g.min())
    m = _flat(1.0 / c ** 2)
    acq = Acquisition(top_row_sources(n, 64), surface_receivers(32))
    return Workload("mixed_256", n, n, 1.0, 1.0, 5.0 * np.arange(1, 9), m, acq)


def config_hypergrad(seed=4, n_models=32):
    """Batched hypergradient: n_models layered models, model k on an n x n grid with
    n = 96 + 32 (k mod 6); omega in {3, 9, 18, 36}; crosswell geometry with N_s in
    [16, 64] sources on the column nearest x = 0.05 and 24 receivers at x = 0.95,
    z ~ U(0.05, 0.95)."""
    rng = np.random.default_rng(seed)
    n_src = int(rng.integers(16, 65))
    rec_z = rng.uniform(0.05, 0.95, 24)
    models = []
    for k in range(n_models):
        n = 96 + 32 * (k % 6)
        h = 1.0 / (n - 1)
        i_src = int(round(0.05 / h))
        zs = np.round(np.linspace(0.05, 0.95, n_src) / h) * h
        acq = Acquisition(np.stack([np.full(n_src, i_src * h), zs], axis=1),
                          np.stack([np.full(24, 0.95), rec_z], axis=1), rec_w=np.ones(24))
        m_true = layered_velocity(n, n, seed * 1000 + k)
        m_fwi = _flat(gaussian_smooth(m_true.reshape(n, n), 4.0))
        models.append(Workload(f"hyper_model_{k}", n, n, 1.0, 1.0, np.array([3.0, 9.0, 18.0, 36.0]),
                               m_fwi, acq, m_true=m_true, alpha=1e-3, mu=1e-6))
    return models


def config_server(seed=5, sizes=(64, 128, 256), n_models=16, n_freq=16):
    """Solve-server load: per grid size n, n_models velocity models (Gaussian random fields,
    correlation length 0.1, mapped to c in [1.5, 4.5]) on the unit square, each with n_freq
    fixed angular frequencies drawn from U[5, 60] (so that requests can hit cached factors).
    Returns {"sizes", "m": [size][model] -> m, "omegas": [size][model][n_freq]}."""
    rng = np.random.default_rng(seed)
    out = {"sizes": list(sizes), "m": [], "omegas": []}
    for si, n in enumerate(sizes):
        ms, oms = [], []
        for k in range(n_models):
            g = gaussian_random_field(n, n, 0.1, seed * 100000 + si * 1000 + k)
            c = 1.5 + 3.0 * (g - g.min()) / (g.max() - g.min())
            ms.append(_flat(1.0 / c ** 2))
            oms.append(np.sort(rng.uniform(5.0, 60.0, n_freq)))
        out["m"].append(ms)
        out["omegas"].append(oms)
    return out


def server_requests(cfg, count, seed, max_rhs=128):
    """count requests of the solve-server load: grid size uniform over cfg["sizes"] (log-uniform
    n), model uniform, frequency uniform over the model's fixed values, right-hand sides
    log-uniform integer in [1, max_rhs], FP64 or mixed with probability 1/2 each.
    Each request is (size index, model index, omega, prec (0 FP64, 1 mixed), nrhs)."""
    rng = np.random.default_rng(seed)
    n_models = len(cfg["m"][0])
    n_freq = len(cfg["omegas"][0][0])
    reqs = []
    for _ in range(count):
        si = int(rng.integers(len(cfg["sizes"])))
        k = int(rng.integers(n_models))
        om = float(cfg["omegas"][si][k][int(rng.integers(n_freq))])
        nrhs = int(min(max_rhs, max(1, round(float(np.exp(rng.uniform(0.0, np.log(max_rhs))))))))
        reqs.append((si, k, om, int(rng.integers(2)), nrhs))
    return reqs


def poisson_arrivals(count, rate, seed):
    """Arrival times (seconds from the start) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, count))


def tiny_case(nx=8, nz=7, n_omega=2, n_src=2, n_rec=3, seed=0, lx=1.0, lz=0.9):
    """Small random case for pins and parity: random smooth-ish m in [1/4, 1], on-grid
    sources on the top row, off-grid receivers in the interior."""
    rng = np.random.default_rng(seed)
    c = 1.0 + rng.uniform(0.0, 1.0, (nx, nz))
    c = gaussian_smooth(c, 1.0)
    m = _flat(1.0 / c ** 2)
    hx = lx / (nx - 1)
    src_i = rng.choice(np.arange(1, nx - 1), size=n_src, replace=False)
    src = np.stack([src_i * hx, np.zeros(n_src)], axis=1)
    rec = np.stack([rng.uniform(0.1, 0.9, n_rec) * lx, rng.uniform(0.2, 0.9, n_rec) * lz], axis=1)
    g2 = rng.uniform(-0.3, 0.3, (nx, nz))
    m_true = _flat(1.0 / (c * (1.0 + 0.2 * gaussian_smooth(g2, 1.0))) ** 2)
    om = np.sort(rng.uniform(2.0, 8.0, n_omega))
    return Workload(f"tiny_{nx}x{nz}", nx, nz, lx, lz, om, m, Acquisition(src, rec), m_true=m_true,
                    alpha=1e-3, mu=1e-3)
