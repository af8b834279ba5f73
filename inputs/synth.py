"""Seeded synthetic right-hand sides shaped like the paper's charged-defect samples.

This module holds no arithmetic of the solver (no centring, no operator, no
preconditioner): it only draws random charge densities.  It is shared by the
oracle-side tests, the GPU tests and the benchmark so that both sides see the
same inputs.

Arrays are returned in storage order: shape ``(nz, ny, nx)``, C-contiguous,
float64, x fastest -- i.e. the flattening equals the paper's vec() order
(first index fastest, Sec. 2.1).

Recipe (stand-in for the Ferrodo2-generated right-hand sides of Problems 1-3,
which are not available):
  * a defect is a Gaussian blob exp(-|x - c|^2 / (2 sigma^2)) evaluated on the
    grid within +-4 sigma of its centre c ~ U[0, n_l) per axis; on periodic
    axes the distance is the minimum image (the window wraps), elsewhere the
    window is clipped to the grid;
  * ``charge`` mode: each blob is scaled so that its grid sum is +-1;
    ``amplitude`` mode: its peak value is the drawn amplitude;
  * optional i.i.d. N(0, noise_std^2) noise;
  * finally the whole array is scaled to ||eta||_2 = 1 / (number of points),
    the normalisation of the paper's experiments (Sec. 5.2).
"""
from __future__ import annotations

import numpy as np

BC_NAMES = ("P", "D", "N", "DN", "ND")


def _axis_profile(n: int, centre: float, sigma: float, periodic: bool):
    """Indices and 1D Gaussian weights of one blob along one axis."""
    if n == 1:
        return np.zeros(1, dtype=np.int64), np.ones(1)
    half = int(np.ceil(4.0 * sigma))
    lo = int(np.floor(centre)) - half
    idx = np.arange(lo, lo + 2 * half + 2)
    d = idx.astype(np.float64) - centre
    w = np.exp(-0.5 * (d / sigma) ** 2)
    if periodic:
        if len(idx) >= n:  # window wider than the axis: fold all images
            folded = np.zeros(n)
            np.add.at(folded, np.mod(idx, n), w)
            return np.arange(n), folded
        return np.mod(idx, n), w
    keep = (idx >= 0) & (idx < n)
    return idx[keep], w[keep]


def add_defects(out, periodic_xyz, centres_xyz, sigmas, weights, mode: str) -> np.ndarray:
    """Add separable Gaussian blobs to a (nz, ny, nx) array in place (and return it)."""
    nz, ny, nx = out.shape
    for c, s, wgt in zip(centres_xyz, sigmas, weights):
        ix, gx = _axis_profile(nx, c[0], s, periodic_xyz[0])
        iy, gy = _axis_profile(ny, c[1], s, periodic_xyz[1])
        iz, gz = _axis_profile(nz, c[2], s, periodic_xyz[2])
        if mode == "charge":
            total = gx.sum() * gy.sum() * gz.sum()
            scale = wgt / total if total > 0 else 0.0
        elif mode == "amplitude":
            scale = wgt
        else:
            raise ValueError(mode)
        blob = scale * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
        out[np.ix_(iz, iy, ix)] += blob
    return out


def gaussian_defects(shape_zyx, periodic_xyz, centres_xyz, sigmas, weights, mode: str) -> np.ndarray:
    """Sum of separable Gaussian blobs on a (nz, ny, nx) grid."""
    return add_defects(np.zeros(shape_zyx), periodic_xyz, centres_xyz, sigmas, weights, mode)


def scale_to_paper_norm(eta: np.ndarray) -> np.ndarray:
    nrm = np.linalg.norm(eta.ravel())
    if nrm == 0:
        return eta
    return eta * ((1.0 / eta.size) / nrm)


def defect_rhs(nx, ny, nz, bcs, n_defects, sigma, seed, mode="charge", noise_std=0.0, amp_range=(-1.0, 1.0),
               normalize=True):
    """A seeded charged-defect right-hand side.

    ``bcs`` is a triple of BC names (x, y, z); periodic axes use minimum-image
    distances.  ``sigma`` is a float or a (lo, hi) range drawn uniformly per
    defect.  In ``charge`` mode the charges are +-1 with equal probability; in
    ``amplitude`` mode peaks are drawn from U(amp_range).
    """
    rng = np.random.default_rng(seed)
    dims = (nx, ny, nz)
    centres = np.stack([rng.uniform(0.0, d, size=n_defects) for d in dims], axis=1)
    if isinstance(sigma, tuple):
        sig = rng.uniform(sigma[0], sigma[1], size=n_defects)
    else:
        sig = np.full(n_defects, float(sigma))
    if mode == "charge":
        w = np.where(rng.random(n_defects) < 0.5, -1.0, 1.0)
    else:
        w = rng.uniform(amp_range[0], amp_range[1], size=n_defects)
    periodic = tuple(b == "P" for b in bcs)
    eta = gaussian_defects((nz, ny, nx), periodic, centres, sig, w, mode)
    if noise_std > 0:
        eta = eta + rng.normal(0.0, noise_std, size=eta.shape)
    return scale_to_paper_norm(eta) if normalize else eta


def random_field(nx, ny, nz, seed):
    """i.i.d. standard normal field, for operator-level parity tests."""
    return np.random.default_rng(seed).standard_normal((nz, ny, nx))


# ---------------------------------------------------------------------------
# The five workloads (grid, BCs, right-hand-side recipe)
# ---------------------------------------------------------------------------
def workload_2d_dirichlet(seed=0):
    """2D 64x64, Dirichlet on all sides, h = 1: 8 blobs, sigma 3 cells, peak amplitudes U(-1, 1)."""
    bcs = ("D", "D", "D")
    eta = defect_rhs(64, 64, 1, bcs, 8, 3.0, seed, mode="amplitude")
    return dict(name="2d-64x64-DD", nx=64, ny=64, nz=1, bcs=bcs, h=(1.0, 1.0, 1.0), eta=eta, tol=1e-12)


def workload_film_128(seed=0):
    """3D 128x128x64 film, periodic x, y and Dirichlet-Neumann z: 200 defects sigma 1.5, +-1, N(0, 1e-3) noise."""
    bcs = ("P", "P", "DN")
    eta = defect_rhs(128, 128, 64, bcs, 200, 1.5, seed, mode="charge", noise_std=1e-3)
    return dict(name="3d-128x128x64-PPDN", nx=128, ny=128, nz=64, bcs=bcs, h=(1.0, 1.0, 1.0), eta=eta, tol=1e-10)


def workload_cuboid_256(seed=0, nz=128):
    """3D 256x256xnz cuboid, periodic x, y and Neumann-Neumann z (singular): 2000 defects sigma U(1, 4), +-1."""
    bcs = ("P", "P", "N")
    eta = defect_rhs(256, 256, nz, bcs, 2000, (1.0, 4.0), seed, mode="charge")
    return dict(name=f"3d-256x256x{nz}-PPN", nx=256, ny=256, nz=nz, bcs=bcs, h=(1.0, 1.0, 1.0), eta=eta, tol=1e-10)


def batched_specs(seed=0, count=48):
    """48 independent solves: nx, ny in {64,96,128,160}, nz in {32,64,96}, BC per axis from {P,D,N,DN,ND},
    1-8 right-hand sides each (film-style defects)."""
    rng = np.random.default_rng(seed)
    specs = []
    for s in range(count):
        nx = int(rng.choice([64, 96, 128, 160]))
        ny = int(rng.choice([64, 96, 128, 160]))
        nz = int(rng.choice([32, 64, 96]))
        bcs = tuple(str(rng.choice(BC_NAMES)) for _ in range(3))
        nrhs = int(rng.integers(1, 9))
        specs.append(dict(nx=nx, ny=ny, nz=nz, bcs=bcs, nrhs=nrhs, seed=int(rng.integers(0, 2**31))))
    return specs


def batched_rhs(spec, r):
    """Right-hand side number r of one batched solve."""
    n_def = max(8, (spec["nx"] * spec["ny"] * spec["nz"]) // 5000)
    return defect_rhs(spec["nx"], spec["ny"], spec["nz"], spec["bcs"], n_def, 1.5, spec["seed"] + 7919 * r,
                      mode="charge", noise_std=1e-3)


class ServingSession:
    """One simulated domain-structure sample issuing a Poisson solve per time step.

    Fixed grid and BCs; its own defect set.  Each step redraws the positions of
    1% of the defects (at least one), as a slowly evolving charge distribution.
    """

    def __init__(self, seed, nx, ny, nz, bcs, n_defects=200, sigma=1.5):
        self.rng = np.random.default_rng(seed)
        self.nx, self.ny, self.nz, self.bcs = nx, ny, nz, bcs
        self.sigma = sigma
        dims = (nx, ny, nz)
        self.centres = np.stack([self.rng.uniform(0.0, d, size=n_defects) for d in dims], axis=1)
        self.charges = np.where(self.rng.random(n_defects) < 0.5, -1.0, 1.0)

    def step(self):
        """Move 1% of the defects; returns (indices, old centres, new centres) of the moved ones."""
        k = max(1, len(self.charges) // 100)
        idx = self.rng.choice(len(self.charges), size=k, replace=False)
        old = self.centres[idx].copy()
        dims = (self.nx, self.ny, self.nz)
        for d in range(3):
            self.centres[idx, d] = self.rng.uniform(0.0, dims[d], size=k)
        return idx, old, self.centres[idx].copy()

    def rhs(self):
        periodic = tuple(b == "P" for b in self.bcs)
        eta = gaussian_defects((self.nz, self.ny, self.nx), periodic, self.centres,
                               np.full(len(self.charges), self.sigma), self.charges, "charge")
        return scale_to_paper_norm(eta)

    def paper_scale(self):
        """Factor that brings the current field to the paper's norm ||eta|| = 1/N (kept for later steps)."""
        periodic = tuple(b == "P" for b in self.bcs)
        eta = gaussian_defects((self.nz, self.ny, self.nx), periodic, self.centres,
                               np.full(len(self.charges), self.sigma), self.charges, "charge")
        nrm = np.linalg.norm(eta.ravel())
        return (1.0 / eta.size) / nrm if nrm > 0 else 1.0

    def apply_moves(self, buf, moves, scale):
        """Update a field in place for the moves returned by step(): the moved defects' blobs are taken
        away at their old centres and added at the new ones, with charges times `scale`."""
        idx, old, new = moves
        periodic = tuple(b == "P" for b in self.bcs)
        sig = np.full(len(idx), self.sigma)
        add_defects(buf, periodic, old, sig, -scale * self.charges[idx], "charge")
        add_defects(buf, periodic, new, sig, scale * self.charges[idx], "charge")
        return buf


def serving_sessions(seed=0, count=16):
    """16 sessions with grids nx, ny in {64..256 step 32}, nz in {32..192 step 32} and random BCs."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(count):
        nx = int(rng.choice(np.arange(64, 257, 32)))
        ny = int(rng.choice(np.arange(64, 257, 32)))
        nz = int(rng.choice(np.arange(32, 193, 32)))
        bcs = tuple(str(rng.choice(BC_NAMES)) for _ in range(3))
        out.append(ServingSession(int(rng.integers(0, 2**31)), nx, ny, nz, bcs))
    return out


def poisson_arrivals(rate_hz, count, seed=0):
    """Seeded exponential inter-arrival times (seconds from start)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=count))
