"""Seeded synthetic inputs (atmospheres and quadrature sizes) for the PORTA hot path.

This module only builds inputs: model-atmosphere arrays and problem sizes.
It holds none of the method's arithmetic (no quadratures, no transfer, no
statistical equilibrium) and is shared by the tests, the oracle runs and the
benchmark so that both sides see identical inputs.

Workloads (the paper's FAL-C / Ca II and Ly-alpha models are not available;
synthetic atmospheres of comparable scale stand in for them):

* ``plane_parallel_box``  16x16x32 unpolarized two-level atom (eps = 1e-2, B = 1),
  exponential opacity with an optional horizontal modulation.
* ``random_box``          polarized two-level atom (Jl=0 -> Ju=1), 64^3 by default,
  log-normal Planck function, opacity and magnetic-field strength, isotropic
  field directions and a Gaussian random vertical velocity.
* ``batched_boxes``       256 boxes of uneven size with the random-box physics.
* ``multilevel_atom`` / ``multilevel_box``  five-level atom (J = 0, 1, 2, 1, 2) with
  four lines, seeded Einstein A and collisional destruction probabilities, in a
  random atmosphere with the random-box statistics (temperature instead of a
  Planck function: the lines have different Planck functions).

Voxel arrays are float64 with shape (nz, ny, nx); index k = 0 is the bottom.
"""
import numpy as np

H_KM = 100.0          # opacity scale height
L_KM = 800.0          # horizontal period
TAU_TOP, TAU_BOT = 1e-4, 1e3


def log_tau_heights(nz, h=H_KM, tau_top=TAU_TOP, tau_bot=TAU_BOT):
    """Heights z_k (km, increasing upward) of nz levels log-spaced in the
    line-centre optical depth tau = exp(-z/h) between tau_bot (k=0) and tau_top."""
    tau = np.geomspace(tau_bot, tau_top, nz)
    return -h * np.log(tau)


def exponential_opacity(z, h=H_KM):
    """chi(z) = exp(-z/h)/h, so that the vertical line-centre optical depth is exp(-z/h)."""
    return np.exp(-z / h) / h


def random_field(rng, shape, slope=-11.0 / 3.0):
    """Standardized Gaussian random field with power spectrum k^slope (k = 0 removed),
    generated on (nx, ny, 2 nz) with periodic FFTs and cropped to nz levels."""
    nz, ny, nx = shape
    gz = 2 * nz
    noise = rng.standard_normal((gz, ny, nx))
    f = np.fft.fftn(noise)
    kz = np.fft.fftfreq(gz)[:, None, None]
    ky = np.fft.fftfreq(ny)[None, :, None]
    kx = np.fft.fftfreq(nx)[None, None, :]
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(k)
    amp[k > 0] = k[k > 0] ** (slope / 2.0)
    g = np.real(np.fft.ifftn(f * amp))[:nz]
    g = g - g.mean()
    sd = g.std()
    return g / sd if sd > 0 else g


def plane_parallel_box(nx=16, ny=16, nz=32, modulation=0.2, eps=1e-2, bpl=1.0, lx=L_KM, ly=L_KM,
                       tau_top=TAU_TOP, tau_bot=TAU_BOT):
    """Unpolarized two-level test box: chi(x,y,z) = chi(z) (1 + a sin(2 pi x/Lx) cos(2 pi y/Ly))."""
    z = log_tau_heights(nz, tau_top=tau_top, tau_bot=tau_bot)
    x = np.arange(nx) * lx / nx
    y = np.arange(ny) * ly / ny
    mod = 1.0 + modulation * np.sin(2 * np.pi * x / lx)[None, None, :] * np.cos(2 * np.pi * y / ly)[None, :, None]
    chi = exponential_opacity(z)[:, None, None] * mod
    shape = (nz, ny, nx)
    return dict(nx=nx, ny=ny, nz=nz, lx=lx, ly=ly, z=z,
                chi=np.broadcast_to(chi, shape).copy(),
                eps=np.full(shape, eps), bpl=np.full(shape, bpl),
                vel=np.zeros(shape), zeta=0.0, gbar=1.0, bcrit=25.0)


def random_box(nx=64, ny=64, nz=64, seed=0, eps=1e-3, sigma_lnb=0.3, sigma_lnchi=0.2,
               b_median=10.0, sigma_lnbfield=1.0, sigma_v=1.0, lx=L_KM, ly=L_KM,
               zeta=3.5e-4, gbar=1.0, bcrit=25.0, tau_top=TAU_TOP, tau_bot=TAU_BOT):
    """Polarized two-level random atmosphere (all fields seeded from SeedSequence(seed))."""
    shape = (nz, ny, nx)
    ss = np.random.SeedSequence(seed).spawn(5)
    r = [np.random.Generator(np.random.PCG64(s)) for s in ss]
    g1 = random_field(r[0], shape)
    g2 = random_field(r[1], shape)
    g3 = random_field(r[2], shape)
    z = log_tau_heights(nz, tau_top=tau_top, tau_bot=tau_bot)
    chi = exponential_opacity(z)[:, None, None] * np.exp(sigma_lnchi * g2)
    bpl = np.exp(sigma_lnb * g1)
    vel = sigma_v * g3
    strength = b_median * np.exp(sigma_lnbfield * r[3].standard_normal(shape))
    d = r[4].standard_normal(shape + (3,))
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    bvec = strength[..., None] * d
    return dict(nx=nx, ny=ny, nz=nz, lx=lx, ly=ly, z=z, chi=chi,
                eps=np.full(shape, eps), bpl=bpl, vel=vel,
                bx=bvec[..., 0].copy(), by=bvec[..., 1].copy(), bz=bvec[..., 2].copy(),
                zeta=zeta, gbar=gbar, bcrit=bcrit)


def batched_boxes(n=256, seed=0, sizes=(8, 16, 24, 32, 48), nz_range=(16, 64)):
    """n independent random boxes of uneven size: Nx = Ny drawn from `sizes`,
    Nz uniform in nz_range (inclusive); box b uses seed (seed, b)."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed)))
    boxes = []
    for b in range(n):
        nxy = int(rng.choice(sizes))
        nz = int(rng.integers(nz_range[0], nz_range[1] + 1))
        boxes.append(random_box(nxy, nxy, nz, seed=[seed, b]))
    return boxes


# five-level model atom: levels J (lower 0-2, upper 3-4), energies in eV and
# the four lines (upper, lower)
ML_J = (0, 1, 2, 1, 2)
ML_E_EV = (0.0, 1.692, 1.700, 3.123, 3.151)
ML_LINES = ((3, 0), (3, 1), (4, 1), (4, 2))


def multilevel_atom(seed=0, a_range=(1e7, 1e8), eps_range=(1e-4, 1e-2), J=ML_J, E=ML_E_EV, lines=ML_LINES):
    """Einstein A (s^-1) and collisional destruction probability eps = C/(A + C)
    per line, both log-uniform in the given ranges (seeded)."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 7])))
    n = len(lines)
    A = np.exp(rng.uniform(np.log(a_range[0]), np.log(a_range[1]), n))
    eps = np.exp(rng.uniform(np.log(eps_range[0]), np.log(eps_range[1]), n))
    return dict(J=np.array(J, dtype=np.int64), E=np.array(E, dtype=np.float64),
                lines=np.array(lines, dtype=np.int64), A=A, eps=eps)


def multilevel_box(nx=128, ny=128, nz=96, seed=0, kT0=0.5, sigma_lnt=0.05, sigma_lnchi=0.2, b_median=30.0,
                   sigma_lnbfield=1.0, sigma_v=1.0, lx=L_KM, ly=L_KM, tau_top=TAU_TOP, tau_bot=TAU_BOT):
    """Random atmosphere for the multilevel atom: the random-box fields with kT
    (eV) = kT0 exp(sigma_lnt g1) in place of the Planck function (sigma_lnt = 0.05
    gives the strongest line's Planck function a log-spread near 0.3, as in the
    random box), chi = the opacity scale (line-centre opacity of the reference
    line with every atom in its lower level), vel and the field B."""
    a = random_box(nx, ny, nz, seed=seed, sigma_lnchi=sigma_lnchi, b_median=b_median,
                   sigma_lnbfield=sigma_lnbfield, sigma_v=sigma_v, lx=lx, ly=ly, tau_top=tau_top, tau_bot=tau_bot)
    g1 = np.log(a.pop("bpl")) / 0.3
    a["kT"] = kT0 * np.exp(sigma_lnt * g1)
    a.pop("eps")
    return a


# problem sizes of the benchmarked configurations
CONFIGS = {
    # name: (atmosphere factory kwargs, model, n_mu per hemisphere, n_chi, n_nu)
    "plain16x16x32": dict(model=0, n_mu=3, n_chi=8, n_nu=11),
    "pol64": dict(model=1, n_mu=5, n_chi=16, n_nu=21),
    "batched256": dict(model=1, n_mu=4, n_chi=10, n_nu=21),
    "ml128": dict(model=2, n_mu=5, n_chi=16, n_nu=31),
}


def emergent_directions():
    """Outgoing lines of sight of the differentiation workload: the vertical and
    four oblique rays (mu = 0.5 at azimuths 0, pi/2, pi, 3 pi/2)."""
    mu = np.array([1.0, 0.5, 0.5, 0.5, 0.5])
    az = np.array([0.0, 0.0, 0.5 * np.pi, np.pi, 1.5 * np.pi])
    return mu, az
