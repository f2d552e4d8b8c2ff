"""Seeded synthetic inputs for the BLINK dirty-image path.

This module is the ONLY code shared between the oracle side (tests) and the
GPU side (tests, bench).  It holds none of the imaging method's arithmetic:
no cell assignment, no gridding, no weighting, no Fourier transform of a grid.
It simulates what a correlator would deliver -- antenna layouts, a point-source
sky, model visibilities V = sum_s S_s exp(-2 pi i (u l_s + v m_s)) (the
coplanar zenith form of the van Cittert-Zernike relation, Sec. 4.3 Eq. 5, with
the primary beam and 1/n folded into S) and Gaussian noise.  The simulator
computes its own baseline vectors as nu * (x_j - x_i) / c, independently of
how the method (or the oracle) computes them.

Every generator is seeded.  The workload shapes mirror the paper's
instruments and runs: 128-tile MWA-like arrays (Sec. 3.2, 8128 baselines),
256-antenna SKA-Low/EDA2-like stations (Sec. 3.1, 32640 baselines),
150-180 MHz, 100 ms time steps (Sec. 6) and 180^2 all-sky images (Fig. 2).
They stand in for the EDA2/MWA data sets of the paper, which are not used.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C_LIGHT = 299792458.0  # m/s

NATURAL = 0
UNIFORM = 1


# --------------------------------------------------------------------- arrays
def antennas_grid(side: int, spacing_m: float) -> np.ndarray:
    """side x side antennas on a square grid (a maximally redundant array:
    the shortest spacing repeats side * (side - 1) times per axis)."""
    g = (np.arange(side) - (side - 1) / 2.0) * spacing_m
    x, y = np.meshgrid(g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), np.zeros(side * side)], axis=1)


def antennas_disk(n_ant: int, diameter_m: float, seed: int) -> np.ndarray:
    """Antenna positions uniform in area inside a disk, z = 0 (coplanar)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    r = 0.5 * diameter_m * np.sqrt(rng.random(n_ant))
    th = 2.0 * math.pi * rng.random(n_ant)
    xyz = np.zeros((n_ant, 3), np.float64)
    xyz[:, 0] = r * np.cos(th)
    xyz[:, 1] = r * np.sin(th)
    return xyz


def pairs(n_ant: int):
    """Cross-correlation pairs (i < j) in lexicographic order."""
    i, j = np.triu_indices(n_ant, k=1)
    return i.astype(np.int64), j.astype(np.int64)


def n_baselines(n_ant: int) -> int:
    return n_ant * (n_ant - 1) // 2


# ------------------------------------------------------------------------ sky
@dataclass
class Sky:
    l: np.ndarray
    m: np.ndarray
    flux: np.ndarray


def sky_box(n_src, half_width, fluxes, seed) -> Sky:
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    l = rng.uniform(-half_width, half_width, n_src)
    m = rng.uniform(-half_width, half_width, n_src)
    return Sky(l, m, np.asarray(fluxes, np.float64))


def sky_disk_loguniform(n_src, radius, smin, smax, seed) -> Sky:
    rng = np.random.Generator(np.random.PCG64(seed + 2000))
    r = radius * np.sqrt(rng.random(n_src))
    th = 2.0 * math.pi * rng.random(n_src)
    flux = np.exp(rng.uniform(math.log(smin), math.log(smax), n_src))
    return Sky(r * np.cos(th), r * np.sin(th), flux)


def model_vis(ant_xyz: np.ndarray, freqs_hz, sky: Sky) -> np.ndarray:
    """Noise-free model visibilities, complex128 [C][B]."""
    i, j = pairs(ant_xyz.shape[0])
    dx = ant_xyz[j, 0] - ant_xyz[i, 0]
    dy = ant_xyz[j, 1] - ant_xyz[i, 1]
    out = np.empty((len(freqs_hz), dx.size), np.complex128)
    for c, nu in enumerate(freqs_hz):
        u = dx * (nu / C_LIGHT)
        v = dy * (nu / C_LIGHT)
        ph = np.outer(u, sky.l) + np.outer(v, sky.m)
        out[c] = (np.exp(-2j * math.pi * ph) * sky.flux[None, :]).sum(axis=1)
    return out


def max_uv(ant_xyz: np.ndarray, freq_hz: float) -> float:
    """Largest |u| or |v| (wavelengths) over all baselines, simulator's formula."""
    i, j = pairs(ant_xyz.shape[0])
    d = np.abs(ant_xyz[j, :2] - ant_xyz[i, :2]).max()
    return float(d * freq_hz / C_LIGHT)


# ---------------------------------------------------------------------- noise
def noise(shape, sigma: float, seed: int, device="cpu"):
    """i.i.d. complex Gaussian noise, sigma per real and imaginary part.

    Returns a torch complex64 tensor on ``device`` (torch's Philox/MT streams
    differ between CPU and CUDA, so a test always feeds both sides the same
    tensor rather than regenerating it).
    """
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    re = torch.randn(shape, generator=g, device=device, dtype=torch.float32)
    im = torch.randn(shape, generator=g, device=device, dtype=torch.float32)
    return torch.complex(re, im) * float(sigma)


# -------------------------------------------------------------------- configs
@dataclass
class Workload:
    """A batch of (time step, channel) layers over one antenna array."""
    name: str
    ant_xyz: np.ndarray
    freqs_hz: np.ndarray          # [C]
    n_times: int
    n_px: np.ndarray              # [C] image size per channel
    delta_u: np.ndarray           # [C] cell size (wavelengths) per channel
    weighting: int
    sigma: float
    sky: Sky
    seed: int
    pulse: dict | None = None     # dispersed single pulse (uneven batch)
    gains: np.ndarray | None = None  # per-antenna complex gains
    notes: dict = field(default_factory=dict)

    @property
    def n_ant(self) -> int:
        return self.ant_xyz.shape[0]

    @property
    def n_chan(self) -> int:
        return len(self.freqs_hz)

    @property
    def n_baselines(self) -> int:
        return n_baselines(self.n_ant)

    @property
    def n_layers(self) -> int:
        return self.n_times * self.n_chan

    def layers(self, times=None, chans=None):
        """Layer descriptors (dicts) for a (time, channel) sub-batch.

        Layer order is time-major, channel-minor; vis_offset indexes the full
        [T][C][B] cube; out_offset packs the selected images contiguously.
        """
        times = range(self.n_times) if times is None else times
        chans = range(self.n_chan) if chans is None else chans
        B = self.n_baselines
        out = []
        off = 0
        for t in times:
            for c in chans:
                n = int(self.n_px[c])
                out.append(dict(n_px=n, weighting=self.weighting, freq_hz=float(self.freqs_hz[c]),
                                delta_u=float(self.delta_u[c]),
                                vis_offset=int((t * self.n_chan + c) * B), out_offset=off,
                                t=int(t), c=int(c)))
                off += n * n
        return out

    def clean_vis(self) -> np.ndarray:
        """Noise-free visibilities per channel, complex128 [C][B] (gains applied)."""
        mv = model_vis(self.ant_xyz, self.freqs_hz, self.sky)
        if self.gains is not None:
            i, j = pairs(self.n_ant)
            mv = mv * (self.gains[i] * np.conj(self.gains[j]))[None, :]
        return mv

    def pulse_flux(self) -> np.ndarray:
        """[T][C] flux of the dispersed pulse (zero outside its arrival step)."""
        p = self.pulse
        nu_top = self.freqs_hz.max() / 1e9
        delay = 4.148808e-3 * p["dm"] * ((self.freqs_hz / 1e9) ** -2 - nu_top ** -2)
        t_arr = p["t0"] + np.rint(delay / p["dt_s"]).astype(np.int64)
        f = np.zeros((self.n_times, self.n_chan), np.float64)
        for c in range(self.n_chan):
            if 0 <= t_arr[c] < self.n_times:
                f[t_arr[c], c] = p["flux"]
        return f

    def vis(self, device="cpu", times=None):
        """complex64 torch tensor [T'][C][B] for the selected time steps."""
        import torch

        times = list(range(self.n_times)) if times is None else list(times)
        B = self.n_baselines
        if self.pulse is None:
            cv = torch.as_tensor(self.clean_vis().astype(np.complex64), device=device)
            out = torch.empty((len(times), self.n_chan, B), dtype=torch.complex64, device=device)
            for k, t in enumerate(times):
                out[k] = cv
        else:
            unit = Sky(self.sky.l, self.sky.m, np.ones_like(self.sky.flux))
            ph = model_vis(self.ant_xyz, self.freqs_hz, unit)  # unit-flux phase pattern
            ph = torch.as_tensor(ph.astype(np.complex64), device=device)
            pf = torch.as_tensor(self.pulse_flux()[times].astype(np.float32), device=device)
            out = pf[:, :, None].to(torch.complex64) * ph[None]
        if self.sigma > 0:
            for k, t in enumerate(times):
                out[k] += noise((self.n_chan, B), self.sigma, self.seed * 1000003 + t, device)
        return out


def _uniform_channels(f_lo, f_hi, n):
    bw = (f_hi - f_lo) / n
    return f_lo + (np.arange(n) + 0.5) * bw


def _du_fill(ant_xyz, f_top, n_px):
    """Cell size that maps the longest baseline at the top frequency to N/2-1."""
    return max_uv(ant_xyz, f_top) / (n_px / 2 - 1)


def single_image(seed=0) -> Workload:
    """One 256^2 natural-weighted image of a 128-antenna 3 km array at 160 MHz."""
    xyz = antennas_disk(128, 3000.0, seed)
    f = np.array([160e6])
    n = np.array([256])
    sky = sky_box(3, 0.5, [1.0, 0.5, 0.2], seed)
    return Workload("single_image_256", xyz, f, 1, n,
                    np.array([_du_fill(xyz, f.max(), 256)]), NATURAL, 0.1, sky, seed)


def station_batch(seed=0, n_times=1000) -> Workload:
    """Station, 1000 steps x 32 channels, 180^2 all-sky, uniform weighting."""
    xyz = antennas_disk(256, 38.0, seed)
    f = _uniform_channels(150e6, 180e6, 32)
    sky = sky_disk_loguniform(20, 1.0, 1.0, 10.0, seed)
    return Workload("station_batch_180", xyz, f, n_times, np.full(32, 180),
                    np.full(32, 0.5), UNIFORM, 1.0, sky, seed)


def uneven_batch(seed=0, n_times=100) -> Workload:
    """128-antenna 3 km array, 768 channels, sizes 128..1024 by channel group."""
    xyz = antennas_disk(128, 3000.0, seed)
    f = _uniform_channels(150e6, 180e6, 768)
    sizes = np.array([128, 256, 512, 1024])[(np.arange(768) // 96) % 4]
    du = np.array([_du_fill(xyz, f.max(), int(n)) for n in sizes])
    sky = sky_box(1, 0.5, [5.0], seed)
    pulse = dict(flux=5.0, dm=100.0, t0=20, dt_s=0.1)
    w = Workload("uneven_batch_pulse", xyz, f, n_times, sizes, du, NATURAL, 1.0, sky, seed,
                 pulse=pulse)
    return w


def station_512(seed=0, n_times=2000) -> Workload:
    """Station, 512^2 images, 2000 steps x 16 channels, 50 sources over 1e-3..10 Jy."""
    xyz = antennas_disk(256, 38.0, seed)
    f = _uniform_channels(150e6, 180e6, 16)
    sky = sky_disk_loguniform(50, 1.0, 1e-3, 10.0, seed)
    return Workload("station_512", xyz, f, n_times, np.full(16, 512), np.full(16, 0.5),
                    NATURAL, 0.1, sky, seed)


def station_gains(seed=0, n_times=100) -> Workload:
    """Station, 1024^2 images, 100 steps x 8 channels, gain-corrupted model."""
    xyz = antennas_disk(256, 38.0, seed)
    f = _uniform_channels(150e6, 180e6, 8)
    sky = sky_disk_loguniform(20, 1.0, 1.0, 10.0, seed)
    rng = np.random.Generator(np.random.PCG64(seed + 3000))
    amp = np.abs(rng.normal(1.0, 0.1, 256))
    ph = rng.uniform(-math.pi, math.pi, 256)
    g = amp * np.exp(1j * ph)
    return Workload("station_gains_1024", xyz, f, n_times, np.full(8, 1024),
                    np.full(8, 0.5), NATURAL, 0.0, sky, seed, gains=g)


WORKLOADS = {"single_image": single_image, "station_batch": station_batch,
             "uneven_batch": uneven_batch, "station_512": station_512, "station_gains": station_gains}
