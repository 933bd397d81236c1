"""Seeded synthetic inputs for the Skyrme-DFT iteration.

This module is the only code shared by the CPU oracle (``oracle/``) and the
CUDA path: it draws the random numbers and builds the trial states and
initial densities, and it holds none of the method's arithmetic (no h,
no damping, no densities of states, no mean fields, no energies).  Both
sides receive the arrays it returns and do everything else themselves.

Layouts (NumPy, C order):
  * spinors   ``psi[I, 2, nz, ny, nx]`` complex128, x fastest.  Component 0
    is spin up, 1 is spin down (Sec. 3.1: ``psi(V, A)`` with V = nx*ny*nz*2).
  * fields    ``f[nz, ny, nx]`` float64.

Workload recipes (Sec. 5.1 and the configurations the benchmarks use):
  * grid spacing 1 fm, cubic periodic boxes, mean densities about
    0.03 fm^-3, proton fraction 0.3-0.5 (the pasta regime of Sec. 1, 5.1);
  * trial states are plane waves for periodic systems (Sec. 2.2), optionally
    with seeded complex Gaussian noise or as seeded random superpositions;
  * initial densities are seeded Gaussian blobs or Fermi-profile pasta
    shapes (sphere, rod, slab: Sec. 1), with a Thomas-Fermi kinetic density.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

# Published SLy4 parameter set (Chabanat et al., Nucl. Phys. A 635 (1998) 231).
# The paper fits "C_q^i" to experiment (Eq. Skyrme) without printing values;
# these are the inputs both the oracle and the CUDA path receive.
SLY4 = dict(
    t0=-2488.91, t1=486.82, t2=-546.39, t3=13777.0,
    x0=0.834, x1=-0.344, x2=-1.0, x3=1.354,
    alpha=1.0 / 6.0, W0=123.0,
    hb2m_n=20.73553, hb2m_p=20.73553,
    e2=1.439964,
)


@dataclass
class Workload:
    """One synthetic workload: box, particle numbers and iteration knobs."""
    name: str
    grid: tuple            # (nx, ny, nz)
    dx: tuple              # fm
    N: int                 # neutrons
    Z: int                 # protons
    coulomb: bool = False
    twist: tuple = (0.0, 0.0, 0.0)
    x0: float = 0.45       # damping step size (Eq. dampstep, delta)
    E0: float = 100.0      # MeV (Eq. dampstep)
    maxit: int = 300
    tol: float = 1e-6      # MeV per nucleon, |E_n/A - E_{n-1}/A|
    init: str = "noisy_plane_waves"   # or "blobs" / "pasta_<shape>"
    noise: float = 0.1
    seed: int = 1001
    nblob: int = 6
    blob_sigma: float = 2.0
    params: dict = field(default_factory=lambda: dict(SLY4))

    def as_dict(self):
        return asdict(self)


def _counts(L3, density=0.03, pfrac=0.3):
    A = int(round(density * L3))
    Z = int(math.floor(pfrac * A + 0.5))
    return A - Z, Z


WORKLOADS = {
    # 16^3, 16 n + 16 p, no Coulomb, noisy plane-wave shells, 300 iterations.
    "sly4_16cubed_16n16p_fp64": Workload(
        name="sly4_16cubed_16n16p_fp64", grid=(16, 16, 16), dx=(1.0, 1.0, 1.0),
        N=16, Z=16, coulomb=False, maxit=300, init="noisy_plane_waves",
        noise=0.1, seed=1001),
    # 24^3, 280 n + 120 p (0.029 fm^-3), FFT-Poisson Coulomb, blob densities
    # and random plane-wave superpositions, 500 iterations.
    "sly4_24cubed_280n120p_coulomb_fp64": Workload(
        name="sly4_24cubed_280n120p_coulomb_fp64", grid=(24, 24, 24),
        dx=(1.0, 1.0, 1.0), N=280, Z=120, coulomb=True, maxit=500,
        init="blobs", seed=1002),
    # 32^3, 700 n + 300 p (precision form; FP32 spinors).
    "sly4_32cubed_700n300p": Workload(
        name="sly4_32cubed_700n300p", grid=(32, 32, 32), dx=(1.0, 1.0, 1.0),
        N=700, Z=300, coulomb=True, maxit=500, init="blobs", seed=1003),
    # The paper's production shapes (Sec. 5, Tables 2-3): A = 6000 (3000 n +
    # 3000 p) in a 32^3 or 48^3 box, dx = 1 fm.
    "sly4_32cubed_3000n3000p": Workload(
        name="sly4_32cubed_3000n3000p", grid=(32, 32, 32), dx=(1.0, 1.0, 1.0),
        N=3000, Z=3000, coulomb=True, maxit=500, init="blobs", seed=1006),
    "sly4_48cubed_3000n3000p": Workload(
        name="sly4_48cubed_3000n3000p", grid=(48, 48, 48), dx=(1.0, 1.0, 1.0),
        N=3000, Z=3000, coulomb=True, maxit=500, init="blobs", seed=1007),
    # Learned-form scale (64^3, 8000 nucleons at 0.03 fm^-3, proton fraction
    # 0.3, FP32 spinors): blob densities; the states are seeded noisy plane
    # waves made on the device (noisy_plane_waves_device), 47 GB of FP64 host
    # arrays being too much to build and copy for a benchmark.
    "sly4_64cubed_5600n2400p": Workload(
        name="sly4_64cubed_5600n2400p", grid=(64, 64, 64), dx=(1.0, 1.0, 1.0),
        N=5600, Z=2400, coulomb=True, maxit=500, init="blobs", noise=0.1, seed=1008),
    # Small 8^3 case for the brute-force pins.
    "sly4_8cubed_4n4p": Workload(
        name="sly4_8cubed_4n4p", grid=(8, 8, 8), dx=(1.0, 1.0, 1.0),
        N=4, Z=4, coulomb=False, maxit=400, init="noisy_plane_waves",
        noise=0.1, seed=1000),
}


def batched_workloads(count=64, seed=1004):
    """Uneven-size twisted instances: grid [16, 20, 24][i mod 3], 0.03 fm^-3,
    proton fraction 0.3, twist drawn uniformly from [-pi, pi)^3."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = (16, 20, 24)[i % 3]
        N, Z = _counts(float(n) ** 3)
        th = tuple(float(v) for v in rng.uniform(-np.pi, np.pi, size=3))
        out.append(Workload(name=f"batched_{i}_{n}cubed", grid=(n, n, n),
                            dx=(1.0, 1.0, 1.0), N=N, Z=Z, twist=th,
                            init="blobs", seed=seed * 1000 + i))
    return out


# --------------------------------------------------------------------------
# Plane-wave basis (trial states for periodic systems, Sec. 2.2)
# --------------------------------------------------------------------------

def plane_wave_labels(grid, dx, count):
    """The ``count`` lowest spin plane waves of the box.

    Ordered by |k|^2 (k_j = 2 pi m_j / L_j, m_j in [-n_j/2, n_j/2)), then
    lexicographically by (m_x, m_y, m_z), spin up before spin down.
    Returns a list of (mx, my, mz, s)."""
    nx, ny, nz = grid
    L = [grid[i] * dx[i] for i in range(3)]
    ms = []
    for mx in range(-(nx // 2), nx - nx // 2):
        for my in range(-(ny // 2), ny - ny // 2):
            for mz in range(-(nz // 2), nz - nz // 2):
                k2 = ((mx / L[0]) ** 2 + (my / L[1]) ** 2 + (mz / L[2]) ** 2)
                ms.append((round(k2, 12), mx, my, mz))
    ms.sort()
    labels = []
    for _, mx, my, mz in ms:
        for s in (0, 1):
            labels.append((mx, my, mz, s))
            if len(labels) == count:
                return labels
    raise ValueError("grid too small for the requested number of plane waves")


def plane_wave_states(grid, dx, labels):
    """e^{i k.r} / sqrt(L^3) times the spin basis vector, on x_a = a*dx."""
    nx, ny, nz = grid
    L = [grid[i] * dx[i] for i in range(3)]
    vol = L[0] * L[1] * L[2]
    x = np.arange(nx) * dx[0]
    y = np.arange(ny) * dx[1]
    z = np.arange(nz) * dx[2]
    out = np.zeros((len(labels), 2, nz, ny, nx), dtype=np.complex128)
    for a, (mx, my, mz, s) in enumerate(labels):
        px = np.exp(2j * np.pi * mx * x / L[0])
        py = np.exp(2j * np.pi * my * y / L[1])
        pz = np.exp(2j * np.pi * mz * z / L[2])
        out[a, s] = (pz[:, None, None] * py[None, :, None] * px[None, None, :]) / math.sqrt(vol)
    return out


def noisy_plane_waves(grid, dx, I, amp, rng):
    """Lowest I plane waves plus amp*(xi_re + i xi_im)/sqrt(2 L^3) per voxel
    and spin component (xi standard normal).  Not orthonormal."""
    labels = plane_wave_labels(grid, dx, I)
    psi = plane_wave_states(grid, dx, labels)
    vol = float(np.prod([grid[i] * dx[i] for i in range(3)]))
    noise = rng.standard_normal(psi.shape) + 1j * rng.standard_normal(psi.shape)
    return psi + amp * noise / math.sqrt(2.0 * vol)


def noisy_plane_waves_device(grid, dx, I, amp, seed, device, dtype):
    """The recipe of noisy_plane_waves (lowest I spin plane waves
    e^{i k.r}/sqrt(L^3) plus amp (xi_re + i xi_im)/sqrt(2 L^3), xi standard
    normal) built on a CUDA device with torch's generator seeded by ``seed``
    (another random stream than NumPy's), in chunks of states; ``dtype``
    torch.complex64 or complex128.  Not orthonormal."""
    import torch
    labels = plane_wave_labels(grid, dx, I)
    nx, ny, nz = grid
    L = [grid[i] * dx[i] for i in range(3)]
    vol = L[0] * L[1] * L[2]
    rdt = torch.float64
    x = torch.arange(nx, device=device, dtype=rdt) * dx[0]
    y = torch.arange(ny, device=device, dtype=rdt) * dx[1]
    z = torch.arange(nz, device=device, dtype=rdt) * dx[2]
    gen = torch.Generator(device=device).manual_seed(int(seed))
    out = torch.empty((I, 2, nz, ny, nx), dtype=dtype, device=device)
    chunk = 64
    for a0 in range(0, I, chunk):
        lab = labels[a0:a0 + chunk]
        m = torch.tensor([[l[0], l[1], l[2]] for l in lab], device=device, dtype=rdt)
        sp = torch.tensor([l[3] for l in lab], device=device)
        phx = torch.exp(2j * math.pi * m[:, 0, None] * x[None, :] / L[0])
        phy = torch.exp(2j * math.pi * m[:, 1, None] * y[None, :] / L[1])
        phz = torch.exp(2j * math.pi * m[:, 2, None] * z[None, :] / L[2])
        pw = (phz[:, :, None, None] * phy[:, None, :, None] * phx[:, None, None, :]) / math.sqrt(vol)
        n = len(lab)
        # complex normal with unit total variance = (xi_re + i xi_im) / sqrt(2)
        noise = torch.randn((n, 2, nz, ny, nx), dtype=torch.complex128, device=device, generator=gen)
        blk = amp * noise / math.sqrt(vol)
        idx = torch.arange(n, device=device)
        blk[idx, sp] += pw
        out[a0:a0 + n] = blk.to(dtype)
    return out


def random_superpositions(grid, dx, I, rng):
    """Each state a seeded complex-normal combination of the 2I lowest spin
    plane waves e^{i k.r}/sqrt(L^3) (the same functions as plane_wave_states),
    synthesised by one inverse FFT per state from its coefficients placed on
    the FFT grid.  Not orthonormal."""
    labels = plane_wave_labels(grid, dx, 2 * I)
    c = rng.standard_normal((I, 2 * I)) + 1j * rng.standard_normal((I, 2 * I))
    nx, ny, nz = grid
    L3 = float(np.prod([grid[i] * dx[i] for i in range(3)]))
    spec = np.zeros((I, 2, nz, ny, nx), dtype=np.complex128)
    for j, (mx, my, mz, s) in enumerate(labels):
        spec[:, s, mz % nz, my % ny, mx % nx] += c[:, j]
    return np.fft.ifftn(spec, axes=(2, 3, 4)) * (nx * ny * nz / np.sqrt(L3))


# --------------------------------------------------------------------------
# Initial densities
# --------------------------------------------------------------------------

def _periodic_distance2(grid, dx, centre):
    nx, ny, nz = grid
    L = [grid[i] * dx[i] for i in range(3)]
    coords = [np.arange(grid[i]) * dx[i] for i in range(3)]
    d2 = np.zeros((nz, ny, nx))
    for i, shape in ((0, (1, 1, nx)), (1, (1, ny, 1)), (2, (nz, 1, 1))):
        d = coords[i] - centre[i]
        d = d - L[i] * np.round(d / L[i])
        d2 = d2 + (d ** 2).reshape(shape)
    return d2


def thomas_fermi_tau(rho):
    """(3/5)(3 pi^2)^{2/3} rho^{5/3}: the initial kinetic-density guess."""
    return 0.6 * (3.0 * np.pi ** 2) ** (2.0 / 3.0) * np.maximum(rho, 0.0) ** (5.0 / 3.0)


def blob_densities(grid, dx, N, Z, nblob, sigma, rng):
    """Sum of nblob periodic Gaussian blobs at seeded uniform centres, scaled
    so that dx^3 * sum(rho_q) = N_q.  Returns rho[2], tau[2] (Thomas-Fermi)."""
    L = [grid[i] * dx[i] for i in range(3)]
    dV = dx[0] * dx[1] * dx[2]
    centres = rng.uniform(0.0, 1.0, size=(nblob, 3)) * np.array(L)
    shape = np.zeros((grid[2], grid[1], grid[0]))
    for c in centres:
        shape += np.exp(-_periodic_distance2(grid, dx, c) / (2.0 * sigma ** 2))
    shape = shape + 1e-3 * shape.max()          # keep a dilute gas everywhere
    shape = shape / (shape.sum() * dV)
    rho = np.stack([N * shape, Z * shape])
    return rho, thomas_fermi_tau(rho)


def pasta_densities(grid, dx, N, Z, kind):
    """Fermi-profile pasta shapes centred in the box: 'sphere' (R = 5 fm),
    'rod' along z (R = 4 fm) or 'slab' normal to z (half width 4 fm), with
    diffuseness 0.5 fm, scaled to N and Z."""
    L = [grid[i] * dx[i] for i in range(3)]
    dV = dx[0] * dx[1] * dx[2]
    c = [0.5 * L[i] for i in range(3)]
    if kind == "sphere":
        d = np.sqrt(_periodic_distance2(grid, dx, c)); R = 5.0
    elif kind == "rod":
        g2 = (grid[0], grid[1], 1)
        d = np.sqrt(_periodic_distance2(g2, dx, c))[0][None, :, :] * np.ones((grid[2], 1, 1)); R = 4.0
    elif kind == "slab":
        z = np.arange(grid[2]) * dx[2] - c[2]
        z = z - L[2] * np.round(z / L[2])
        d = np.abs(z)[:, None, None] * np.ones((1, grid[1], grid[0])); R = 4.0
    else:
        raise ValueError(kind)
    f = 1.0 / (1.0 + np.exp((d - R) / 0.5)) + 1e-3
    f = f / (f.sum() * dV)
    rho = np.stack([N * f, Z * f])
    return rho, thomas_fermi_tau(rho)


def make_inputs(w: Workload, seed=None):
    """Host arrays for one workload.

    Returns dict with ``psi0 = [psi_n, psi_p]`` (raw, NOT orthonormal) and,
    for density-started workloads, ``rho0``/``tau0`` ([2, nz, ny, nx]; the
    initial spin-orbit density is zero).  Seed defaults to ``w.seed``."""
    rng = np.random.default_rng(w.seed if seed is None else seed)
    out = {}
    if w.init == "noisy_plane_waves":
        out["psi0"] = [noisy_plane_waves(w.grid, w.dx, w.N, w.noise, rng),
                       noisy_plane_waves(w.grid, w.dx, w.Z, w.noise, rng)]
    else:
        out["psi0"] = [random_superpositions(w.grid, w.dx, w.N, rng),
                       random_superpositions(w.grid, w.dx, w.Z, rng)]
        if w.init == "blobs":
            rho, tau = blob_densities(w.grid, w.dx, w.N, w.Z, w.nblob, w.blob_sigma, rng)
        elif w.init.startswith("pasta_"):
            rho, tau = pasta_densities(w.grid, w.dx, w.N, w.Z, w.init[6:])
        else:
            raise ValueError(w.init)
        out["rho0"], out["tau0"] = rho, tau
    return out


def random_smooth_field(grid, rng, mean, amp, nmodes=4):
    """A real periodic field: mean + sum of a few seeded low Fourier modes."""
    nx, ny, nz = grid
    z, y, x = np.meshgrid(np.arange(nz) / nz, np.arange(ny) / ny, np.arange(nx) / nx, indexing="ij")
    f = np.full((nz, ny, nx), float(mean))
    for _ in range(nmodes):
        m = rng.integers(-2, 3, size=3)
        ph = rng.uniform(0, 2 * np.pi)
        a = rng.uniform(-1, 1) * amp / nmodes
        f += a * np.cos(2 * np.pi * (m[0] * x + m[1] * y + m[2] * z) + ph)
    return f


def random_spinors(grid, I, rng):
    """Complex standard-normal spinors (no structure), for operator tests."""
    nx, ny, nz = grid
    s = (I, 2, nz, ny, nx)
    return rng.standard_normal(s) + 1j * rng.standard_normal(s)
