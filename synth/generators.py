"""Seeded synthetic workloads shaped like the paper's visible-light and electron data.

The paper's own datasets (optical QPT and USAF data, Sec. 3.1 and Sec. 4.6; the
MoSe2/WS2 and PrScO3 4D-STEM sets, Sec. 3.2 and Sec. 4.1) are not available, so
these generators stand in for them. Each configuration simulates the physical
measurement:

* far field: I_n = |F(P . o_n)|^2 in the detector-centred frame (Eq. 1);
* near field: I_n = |F^-1(F(P . o_n) H)|^2 with the Fresnel transfer function H;
* partial coherence: the coherent intensity is convolved with a normalised
  Gaussian (Eq. 2, the physics, truncated at +-ceil(5 sigma), zero padded);
* temporal coherence (far field): a sum of per-wavelength patterns, each
  rescaled about the detector centre with the wavelength (Sec. 3.1, the
  2 pi / (lambda z) scaling);
* shot noise: one global scale so that the mean pattern holds `dose` counts,
  then Poisson sampling.

Random streams: numpy.random.default_rng(SeedSequence(seed).spawn(4)), used
for the object, the probe, the scan and the noise, in that order.

numpy.fft and scipy.ndimage are used here as library primitives to simulate
the measurement. Nothing computed here is handed to either reconstruction
path except the raw arrays of a `Problem`.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np
from scipy import ndimage

CONFIG_NAMES = {
    0: "far-field plain engine: M=64, K=1, N=100, object 192^2, sigma=1, 1e5 photons",
    1: "far-field 4 modes: M=128, K=4, N=900 Fermat spiral, object 640^2, 5% bandwidth, sigma=1.5, 1e6 photons",
    2: "near-field Fresnel F=10: M=256, K=8, N=256, object 1024^2, sigma=2, 1e5 photons",
    3: "batched: 64 uneven reconstructions, M in {64,128,256}, N in [100,1600], far/near",
    4: "electron 300 kV: M=128, K=1, N=4096, object 256^2, sigma=2, 200 e/pattern",
}


@dataclasses.dataclass
class Problem:
    """One reconstruction problem: measured data, scan, truth and initial state."""

    name: str
    I: np.ndarray  # (N, M, M) float32 measured intensities (far field: DC at (M/2, M/2))
    I_clean: np.ndarray  # (N, M, M) float64 noise-free intensities at the same dose
    positions: np.ndarray  # (N, 2) int32 top-left (row, col) of each object box
    O_true: np.ndarray  # (H, W) complex128
    P_true: np.ndarray  # (M, M) complex128 physical probe
    O0: np.ndarray  # (H, W) complex64 initial object (flat 1)
    P0: np.ndarray  # (K, M, M) complex64 initial probe modes
    params: dict  # engine parameters (keys follow ptycho_params)
    sim_sigma: float  # the blur width used to simulate the data

    @property
    def M(self) -> int:
        return int(self.I.shape[1])

    @property
    def N(self) -> int:
        return int(self.I.shape[0])

    @property
    def K(self) -> int:
        return int(self.P0.shape[0])


# ----------------------------------------------------------------------------------------
# geometry helpers (pinned against the paper's Table 1 and Sec. 3.1 in tests/golden)
# ----------------------------------------------------------------------------------------

def far_field_object_pixel(wavelength: float, z: float, M: int, det_pixel: float) -> float:
    """Real-space pixel of a far-field reconstruction, lambda z / (M dk) (Table 1)."""
    return wavelength * z / (M * det_pixel)


def qpt_phase(wavelength: float, n_index: float, thickness: float) -> float:
    """Phase of the quantitative phase target, 2 pi / lambda (n - 1) d (Sec. 3.1)."""
    return 2.0 * math.pi / wavelength * (n_index - 1.0) * thickness


def electron_wavelength(volts: float) -> float:
    """Relativistic electron wavelength in metres for an accelerating voltage."""
    h = 6.62607015e-34
    m0 = 9.1093837015e-31
    e = 1.602176634e-19
    c = 299792458.0
    return h / math.sqrt(2.0 * m0 * e * volts * (1.0 + e * volts / (2.0 * m0 * c * c)))


# ----------------------------------------------------------------------------------------
# fields
# ----------------------------------------------------------------------------------------

def _grf(rng, shape, corr_len, lo, hi):
    """Gaussian random field: white noise low-passed by a Gaussian, min-max scaled to [lo, hi]."""
    f = ndimage.gaussian_filter(rng.standard_normal(shape), corr_len, mode="wrap")
    f = (f - f.min()) / (f.max() - f.min())
    return lo + (hi - lo) * f


def _radius_grid(M):
    y, x = np.mgrid[0:M, 0:M].astype(np.float64)
    c = (M - 1) / 2.0
    return np.hypot(y - c, x - c), np.arctan2(y - c, x - c)


def _zernike_radial(n, m, rho):
    m = abs(m)
    out = np.zeros_like(rho)
    for s in range((n - m) // 2 + 1):
        coef = ((-1) ** s * math.factorial(n - s)
                / (math.factorial(s) * math.factorial((n + m) // 2 - s) * math.factorial((n - m) // 2 - s)))
        out += coef * rho ** (n - 2 * s)
    return out


def _disc_probe(M, radius, phase=None):
    r, _ = _radius_grid(M)
    p = (r <= radius).astype(np.complex128)
    if phase is not None:
        p = p * np.exp(1j * phase)
    return p


def _intensity_blur(I, sigma):
    """Eq. 2 physics: intensity convolved with a normalised Gaussian, +-ceil(5 sigma), zero padded."""
    if sigma <= 0:
        return I.copy()
    h = int(math.ceil(5 * sigma))
    t = np.arange(-h, h + 1, dtype=np.float64)
    g = np.exp(-t * t / (2 * sigma * sigma))
    g /= g.sum()
    out = ndimage.correlate1d(I, g, axis=-1, mode="constant", cval=0.0)
    return ndimage.correlate1d(out, g, axis=-2, mode="constant", cval=0.0)


def _fresnel_tf(M, F):
    u = np.fft.fftfreq(M) * M
    return np.exp(-1j * np.pi * (u[:, None] ** 2 + u[None, :] ** 2) / (M * F))


def _exit_waves(O, P, positions):
    M = P.shape[-1]
    return np.stack([P * O[y:y + M, x:x + M] for (y, x) in positions])


def _coherent_far(psi):
    return np.abs(np.fft.fftshift(np.fft.fft2(psi), axes=(-2, -1))) ** 2


def _coherent_near(psi, F):
    H = _fresnel_tf(psi.shape[-1], F)
    return np.abs(np.fft.ifft2(np.fft.fft2(psi) * H)) ** 2


def _rescale_about_centre(I, s):
    """Magnify a centred pattern by s about (M/2, M/2), keeping its energy."""
    M = I.shape[-1]
    c = M / 2.0
    y, x = np.mgrid[0:M, 0:M].astype(np.float64)
    coords = np.stack([(y - c) / s + c, (x - c) / s + c])
    out = np.empty_like(I)
    for i in range(I.shape[0]):
        out[i] = ndimage.map_coordinates(I[i], coords, order=1, mode="constant", cval=0.0)
    return out / (s * s)


def _simulate(O, P, positions, geometry, sigma, dose, rng_noise, fresnel_F=10.0, rel_wavelengths=None):
    psi = _exit_waves(O, P, positions)
    if geometry == "far":
        Ic = _coherent_far(psi)
        if rel_wavelengths is not None:
            Ic = sum(_rescale_about_centre(Ic, s) for s in rel_wavelengths) / len(rel_wavelengths)
    else:
        Ic = _coherent_near(psi, fresnel_F)
    Ipc = _intensity_blur(Ic, sigma)
    Ipc = np.maximum(Ipc, 0.0)
    Ipc *= dose / Ipc.sum(axis=(1, 2)).mean()
    I = rng_noise.poisson(Ipc).astype(np.float32)
    return I, Ipc


def _initial_probe(P_design, K, I, geometry, rng):
    """P0 scaled by Parseval to the mean measured energy; extra modes at 10% with a random phase."""
    M = P_design.shape[-1]
    energy = float(np.sum(I, dtype=np.float64)) / I.shape[0]
    target = energy / (M * M) if geometry == "far" else energy
    p = P_design * math.sqrt(target / np.sum(np.abs(P_design) ** 2))
    modes = [p]
    for _ in range(1, K):
        modes.append(0.1 * p * np.exp(1j * rng.uniform(0, 2 * np.pi, size=p.shape)))
    return np.stack(modes).astype(np.complex64)


def _base_params(M, K, N, H, W, geometry, sigma, n_iter, fresnel_F=0.0, windows=()):
    return dict(M=M, K=K, N=N, obj_h=H, obj_w=W, geometry=geometry, blur_domain="amplitude",
                fresnel_F=float(fresnel_F), sigma1=float(sigma), sigma2=float(sigma), kernel_size=11,
                eps_mod=0.0, beta_obj=1.0, beta_probe=1.0, delta_obj=1e-3, delta_probe=1e-3,
                probe_update_start=1, alpha1=1.0, alpha2=0.0, cbar_min=0.01, cbar_max=10.0,
                windows=list(windows), start_iteration=1, n_iter=n_iter)


def _streams(seed):
    return [np.random.default_rng(s) for s in np.random.SeedSequence(seed).spawn(4)]


# ----------------------------------------------------------------------------------------
# configurations
# ----------------------------------------------------------------------------------------

def _cfg0(seed, scan_side=10, obj_side=192, M=64, K=1, dose=1e5, sigma=1.0, geometry="far"):
    r_obj, r_probe, r_scan, r_noise = _streams(seed)
    amp = r_obj.uniform(0.8, 1.0, size=(obj_side, obj_side))
    phase = _grf(r_obj, (obj_side, obj_side), 8.0, 0.0, np.pi)
    O = amp * np.exp(1j * phase)
    radius = 20.0 * M / 64
    r, _ = _radius_grid(M)
    P = _disc_probe(M, radius, 4 * np.pi * (r / radius) ** 2)
    step = 12 * M // 64
    extent = (scan_side - 1) * step + M
    off = (obj_side - extent) // 2
    jit = np.rint(r_scan.uniform(-1, 1, size=(scan_side * scan_side, 2))).astype(int)
    grid = np.array([(off + i * step, off + j * step) for i in range(scan_side) for j in range(scan_side)])
    pos = np.clip(grid + jit, 0, obj_side - M).astype(np.int32)
    I, Ic = _simulate(O, P, pos, geometry, sigma, dose, r_noise, fresnel_F=10.0)
    P0 = _initial_probe(P, K, I, geometry, r_probe)
    prm = _base_params(M, K, len(pos), obj_side, obj_side, geometry, sigma, 50,
                       fresnel_F=10.0 if geometry == "near" else 0.0)
    return Problem("cfg0", I, Ic, pos, O, P, np.ones_like(O, dtype=np.complex64), P0, prm, sigma)


def _cfg1(seed, n_pos=900, obj_side=640, M=128, K=4, dose=1e6, sigma=1.5, mean_step=6.0):
    r_obj, r_probe, r_scan, r_noise = _streams(seed)
    amp = r_obj.uniform(0.8, 1.0, size=(obj_side, obj_side))
    phase = _grf(r_obj, (obj_side, obj_side), 8.0, 0.0, np.pi)
    O = amp * np.exp(1j * phase)
    radius = 40.0 * M / 128
    r, th = _radius_grid(M)
    rho = np.minimum(r / radius, 1.0)
    zphase = np.zeros((M, M))
    for n in range(1, 5):
        for m in range(-n, n + 1, 2):
            c = r_probe.standard_normal()
            ang = np.cos(m * th) if m >= 0 else np.sin(-m * th)
            zphase += c * _zernike_radial(n, m, rho) * ang
    P = _disc_probe(M, radius, zphase)
    P_design = _disc_probe(M, radius)
    golden = np.pi * (3.0 - math.sqrt(5.0))
    c_sp = mean_step / math.sqrt(math.pi)
    i = np.arange(n_pos)
    ry = c_sp * np.sqrt(i) * np.sin(i * golden)
    rx = c_sp * np.sqrt(i) * np.cos(i * golden)
    centre = obj_side / 2.0 - M / 2.0
    pos = np.stack([np.rint(centre + ry), np.rint(centre + rx)], axis=1)
    pos = np.clip(pos, 0, obj_side - M).astype(np.int32)
    rel = [1.0 + d for d in (-0.025, -0.0125, 0.0, 0.0125, 0.025)]
    I, Ic = _simulate(O, P, pos, "far", sigma, dose, r_noise, rel_wavelengths=rel)
    P0 = _initial_probe(P_design, K, I, "far", r_probe)
    prm = _base_params(M, K, len(pos), obj_side, obj_side, "far", sigma, 200)
    return Problem("cfg1", I, Ic, pos, O, P, np.ones_like(O, dtype=np.complex64), P0, prm, sigma)


def _diffuser(rng, M, smooth=3.0):
    screen = _grf(rng, (M, M), smooth, 0.0, 2 * np.pi)
    r, _ = _radius_grid(M)
    apod = np.exp(-(r / (0.4 * M)) ** 8)
    return apod * np.exp(1j * screen), apod


def _cfg2(seed, scan_side=16, obj_side=1024, M=256, K=8, dose=1e5, sigma=2.0, F=10.0, step=20):
    r_obj, r_probe, r_scan, r_noise = _streams(seed)
    amp = _grf(r_obj, (obj_side, obj_side), 8.0, 0.85, 1.0)
    yy, xx = np.mgrid[0:obj_side, 0:obj_side].astype(np.float64)
    th = np.arctan2(yy - obj_side / 2, xx - obj_side / 2)
    phase = 0.5 * (np.sin(36 * th) > 0)
    O = amp * np.exp(1j * phase)
    P, apod = _diffuser(r_probe, M)
    P_design = ndimage.gaussian_filter(P.real, 2.0) + 1j * ndimage.gaussian_filter(P.imag, 2.0)
    extent = (scan_side - 1) * step + M
    off = (obj_side - extent) // 2
    pos = np.array([(off + i * step, off + j * step) for i in range(scan_side) for j in range(scan_side)],
                   dtype=np.int32)
    I, Ic = _simulate(O, P, pos, "near", sigma, dose, r_noise, fresnel_F=F)
    P0 = _initial_probe(P_design, K, I, "near", r_probe)
    prm = _base_params(M, K, len(pos), obj_side, obj_side, "near", sigma, 300, fresnel_F=F)
    return Problem("cfg2", I, Ic, pos, O, P, np.ones_like(O, dtype=np.complex64), P0, prm, sigma)


def _cfg3_member(seed, M, K, N, geometry, sigma, dose=1e5, F=10.0):
    r_obj, r_probe, r_scan, r_noise = _streams(seed)
    step = int(math.ceil(0.15 * M))
    ncol = int(math.ceil(math.sqrt(N)))
    nrow = int(math.ceil(N / ncol))
    side = M + (max(ncol, nrow) - 1) * step
    amp = r_obj.uniform(0.8, 1.0, size=(side, side))
    phase = _grf(r_obj, (side, side), 8.0, 0.0, np.pi)
    O = amp * np.exp(1j * phase)
    if geometry == "far":
        radius = 0.3 * M
        r, _ = _radius_grid(M)
        P = _disc_probe(M, radius, r_probe.uniform(2, 6) * np.pi * (r / radius) ** 2)
        P_design = P
    else:
        P, _ = _diffuser(r_probe, M)
        P_design = ndimage.gaussian_filter(P.real, 2.0) + 1j * ndimage.gaussian_filter(P.imag, 2.0)
    pos = np.array([(i * step, j * step) for i in range(nrow) for j in range(ncol)][:N], dtype=np.int32)
    I, Ic = _simulate(O, P, pos, geometry, sigma, dose, r_noise, fresnel_F=F)
    P0 = _initial_probe(P_design, K, I, geometry, r_probe)
    prm = _base_params(M, K, len(pos), side, side, geometry, sigma, 100,
                       fresnel_F=F if geometry == "near" else 0.0)
    return Problem(f"cfg3[{seed}]", I, Ic, pos, O, P, np.ones_like(O, dtype=np.complex64), P0, prm, sigma)


def cfg3_members(seed=3, count=64, M_choices=(64, 128, 256), N_range=(100, 1600)):
    """Descriptors (M, K, N, geometry, sigma) of the batched configuration's problems."""
    rng = np.random.default_rng(np.random.SeedSequence(seed).spawn(5)[4])
    out = []
    for _ in range(count):
        M = int(rng.choice(M_choices))
        K = int(rng.choice([1, 2, 4]))
        N = int(rng.integers(N_range[0], N_range[1] + 1))
        geometry = "far" if rng.random() < 0.5 else "near"
        sigma = float(rng.uniform(0.5, 3.0))
        out.append((M, K, N, geometry, sigma))
    return out


def _cfg4(seed, scan_side=64, M=128, obj_side=256, dose=200.0, sigma=2.0, dx=0.2e-10, step=2, peak=0.1):
    r_obj, r_probe, r_scan, r_noise = _streams(seed)
    lam = electron_wavelength(300e3)
    # hexagonal lattice of Gaussian phase peaks (`peak` rad, 0.1 by default), sigma 0.3 A, 5% vacancies,
    # random rotation
    a = 3.2e-10 / dx
    s_pk = 0.3e-10 / dx
    rot = r_obj.uniform(0, np.pi / 3)
    a1 = a * np.array([math.cos(rot), math.sin(rot)])
    a2 = a * np.array([math.cos(rot + np.pi / 3), math.sin(rot + np.pi / 3)])
    nmax = int(2 * obj_side / a) + 2
    phase = np.zeros((obj_side, obj_side))
    yy, xx = np.mgrid[0:obj_side, 0:obj_side].astype(np.float64)
    h = int(math.ceil(4 * s_pk))
    for i in range(-nmax, nmax + 1):
        for j in range(-nmax, nmax + 1):
            p = i * a1 + j * a2 + obj_side / 2.0
            if not (-h <= p[0] < obj_side + h and -h <= p[1] < obj_side + h):
                continue
            if r_obj.random() < 0.05:
                continue
            y0, y1 = max(int(p[0]) - h, 0), min(int(p[0]) + h + 1, obj_side)
            x0, x1 = max(int(p[1]) - h, 0), min(int(p[1]) + h + 1, obj_side)
            phase[y0:y1, x0:x1] += peak * np.exp(
                -((yy[y0:y1, x0:x1] - p[0]) ** 2 + (xx[y0:y1, x0:x1] - p[1]) ** 2) / (2 * s_pk * s_pk))
    O = np.exp(1j * phase)
    # defocused probe: 25 mrad aperture, 20 nm defocus
    k = np.fft.fftshift(np.fft.fftfreq(M, d=dx))
    k2 = k[:, None] ** 2 + k[None, :] ** 2
    aperture = (np.sqrt(k2) * lam <= 25e-3).astype(np.float64)
    chi = np.pi * lam * 20e-9 * k2
    P = np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(aperture * np.exp(-1j * chi))))
    pos = np.array([(i * step, j * step) for i in range(scan_side) for j in range(scan_side)], dtype=np.int32)
    I, Ic = _simulate(O, P, pos, "far", sigma, dose, r_noise)
    P0 = _initial_probe(P, 1, I, "far", r_probe)
    prm = _base_params(M, 1, len(pos), obj_side, obj_side, "far", sigma, 200)
    return Problem("cfg4", I, Ic, pos, O, P, np.ones_like(O, dtype=np.complex64), P0, prm, sigma)


def make_problem(cfg: int, seed: Optional[int] = None, **kw) -> Problem:
    """Build configuration `cfg` (0, 1, 2 or 4; 3 via `cfg3_members` + `make_cfg3_member`).

    Keyword arguments shrink or reshape a configuration for tests (scan size,
    probe size, modes, geometry, dose, blur width).
    """
    seed = cfg if seed is None else seed
    if cfg == 0:
        return _cfg0(seed, **kw)
    if cfg == 1:
        return _cfg1(seed, **kw)
    if cfg == 2:
        return _cfg2(seed, **kw)
    if cfg == 4:
        return _cfg4(seed, **kw)
    raise ValueError(f"unknown configuration {cfg}")


def make_cfg3_member(index: int, seed: int = 3, count: int = 64, **kw) -> Problem:
    M, K, N, geometry, sigma = cfg3_members(seed, count)[index]
    kw.setdefault("N", N)
    return _cfg3_member(1000 * seed + index, kw.pop("M", M), kw.pop("K", K), kw.pop("N"),
                        kw.pop("geometry", geometry), kw.pop("sigma", sigma), **kw)
