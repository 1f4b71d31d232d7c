"""Seeded synthetic visibility workloads.

The paper measures on a simulated MeerKAT observation (Merry 2016, Sec. 5),
which is not available here. This module makes seeded stand-ins with the same
structure:
  - visibilities ordered by baseline (Sec. 4), then time, then channel;
  - earth-rotation uv tracks, so consecutive samples of a baseline move
    slowly across the uv plane (the coherence that Romein's algorithm relies
    on, Sec. 2.2);
  - complex Gaussian values and unit weights.

This module only synthesizes inputs. It contains none of the gridding
arithmetic, and both the CUDA path and the FP64 oracle consume what it
returns.

Recipe (all angles in degrees):
  - Antennas are uniform in a disk of radius R: radius R*sqrt(U1), angle
    360*U2. They are coplanar (up = 0).
  - Baselines are all pairs p < q, in (p, q) order. The baseline vector is
    ENU(q) - ENU(p).
  - ENU is converted to equatorial (X, Y, Z) at latitude lat:
    X = -sin(lat) N + cos(lat) U, Y = E, Z = cos(lat) N + sin(lat) U.
  - The hour angle H is uniform over [-span/2, +span/2) in n_times steps, at
    declination dec. Then u = sin H X + cos H Y and
    v = -sin(dec) cos H X + sin(dec) sin H Y + cos(dec) Z. The w term is
    not used.
  - Channel k scales (u, v) by 1 + k/1024.
  - (u, v) is scaled so that max(|u|, |v|) over every channel equals
    0.9 * (G/2 - h - 1) pixels, where h = (S-1)//2.
  - Values are complex N(0, 1) (independent real and imaginary parts),
    complex64. Weights are 1, float32.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

LATITUDE_DEG = -30.7
DECLINATION_DEG = -30.0
HOUR_ANGLE_SPAN_H = 8.0
CHANNEL_STEP = 1.0 / 1024.0


@dataclass
class Workload:
    """One gridding problem: sizes plus the inputs to grid()."""

    name: str
    G: int
    S: int
    oversample: int
    npol: int
    uv: np.ndarray          # [N, 2] float64, grid-pixel units relative to the grid centre
    vis: np.ndarray         # [N, P] complex64
    weights: np.ndarray     # [N] float32
    beta: float = 0.0       # Kaiser-Bessel shape parameter (2.34 * S)
    meta: dict = field(default_factory=dict)

    @property
    def n_vis(self) -> int:
        return int(self.uv.shape[0])


def antenna_layout(n_ant: int, radius_m: float, rng: np.random.Generator) -> np.ndarray:
    """ENU antenna positions [n_ant, 3], uniform in a disk, with up = 0."""
    r = radius_m * np.sqrt(rng.random(n_ant))
    a = 2.0 * np.pi * rng.random(n_ant)
    return np.stack([r * np.cos(a), r * np.sin(a), np.zeros(n_ant)], axis=1)


def cored_layout(n_core: int, r_core_m: float, n_outer: int, r_outer_m: float, rng: np.random.Generator) -> np.ndarray:
    """ENU positions of a dense core (n_core antennas in a disk of r_core_m) plus n_outer out to r_outer_m."""
    return np.concatenate([antenna_layout(n_core, r_core_m, rng), antenna_layout(n_outer, r_outer_m, rng)])


def baseline_pairs(n_ant: int) -> np.ndarray:
    """All (p, q) with p < q, in (p, q) order. Shape [n_ant*(n_ant-1)/2, 2]."""
    p, q = np.triu_indices(n_ant, k=1)
    return np.stack([p, q], axis=1)


def uv_tracks_m(enu: np.ndarray, n_times: int, n_chan: int) -> np.ndarray:
    """Earth-rotation (u, v) in metres, shape [n_bl, n_times, n_chan, 2], channel scaling included."""
    pairs = baseline_pairs(enu.shape[0])
    L = enu[pairs[:, 1]] - enu[pairs[:, 0]]                       # [n_bl, 3] ENU
    lat = np.deg2rad(LATITUDE_DEG)
    dec = np.deg2rad(DECLINATION_DEG)
    X = -np.sin(lat) * L[:, 1] + np.cos(lat) * L[:, 2]
    Y = L[:, 0]
    Z = np.cos(lat) * L[:, 1] + np.sin(lat) * L[:, 2]
    H = np.deg2rad(15.0 * HOUR_ANGLE_SPAN_H * (np.arange(n_times) / n_times - 0.5))
    sH, cH = np.sin(H)[None, :], np.cos(H)[None, :]
    u = sH * X[:, None] + cH * Y[:, None]
    v = -np.sin(dec) * cH * X[:, None] + np.sin(dec) * sH * Y[:, None] + np.cos(dec) * Z[:, None]
    scale = 1.0 + CHANNEL_STEP * np.arange(n_chan)
    uv = np.stack([u, v], axis=-1)                                  # [n_bl, n_t, 2]
    return uv[:, :, None, :] * scale[None, None, :, None]          # [n_bl, n_t, n_chan, 2]


def scale_to_grid(uv_m: np.ndarray, G: int, S: int) -> np.ndarray:
    """Scale so max(|u|,|v|) maps to 0.9*(G/2 - h - 1) pixels. Returns float64 pixels."""
    h = (S - 1) // 2
    m = float(np.max(np.abs(uv_m)))
    return (uv_m * (0.9 * (G / 2 - h - 1) / m)).astype(np.float64)


def gaussian_values(rng: np.random.Generator, n: int, npol: int) -> np.ndarray:
    """Complex N(0,1) values, [n, npol] complex64."""
    z = rng.standard_normal((n, npol, 2), dtype=np.float32)
    return (z[..., 0] + 1j * z[..., 1]).astype(np.complex64)


def observation(name: str, G: int, S: int, oversample: int, npol: int, n_ant: int, radius_m: float,
                n_times: int, n_chan: int, seed: int = 0, limit: int | None = None, layout=None) -> Workload:
    """A baseline-ordered observation: n_bl x n_times x n_chan samples (channel fastest).

    ``layout(rng)`` returns the ENU antenna positions; the default is n_ant uniform in a disk of radius_m.
    """
    rng = np.random.default_rng(seed)
    enu = antenna_layout(n_ant, radius_m, rng) if layout is None else layout(rng)
    assert enu.shape == (n_ant, 3)
    uv = scale_to_grid(uv_tracks_m(enu, n_times, n_chan), G, S).reshape(-1, 2)
    if limit is not None:
        uv = np.ascontiguousarray(uv[:limit])
    n = uv.shape[0]
    vis = gaussian_values(rng, n, npol)
    w = np.ones(n, np.float32)
    return Workload(name, G, S, oversample, npol, uv, vis, w, beta=2.34 * S,
                    meta=dict(n_ant=n_ant, radius_m=radius_m, n_times=n_times, n_chan=n_chan, seed=seed))


def plain_single_pol(seed: int = 0) -> Workload:
    """G=256, S=7, O=8, P=1; 16 antennas in a 2 km disk; 120 bl x 256 t x 1 ch = 30,720 vis."""
    return observation("plain-single-pol G256 S7 O8 P1 30720vis", 256, 7, 8, 1, 16, 1000.0, 256, 1, seed)


def quad_pol(seed: int = 0) -> Workload:
    """G=2048, S=7, O=8, P=4; 64 antennas in an 8 km disk; 2016 bl x 1024 t x 4 ch = 8,257,536 vis."""
    return observation("quad-pol G2048 S7 O8 P4 8257536vis", 2048, 7, 8, 4, 64, 4000.0, 1024, 4, seed)


def precision_single_pol(seed: int = 0) -> Workload:
    """G=4096, S=15, O=16, P=1; 256 antennas in a 16 km disk; 32640 bl x 256 t x 2 ch = 16,711,680 vis."""
    return observation("precision G4096 S15 O16 P1 16711680vis", 4096, 15, 16, 1, 256, 8000.0, 256, 2, seed)


def differentiation(seed: int = 0) -> Workload:
    """G=1024, S=7, O=8, P=1; 64 antennas; the first 1,000,000 of 2016 bl x 497 t."""
    return observation("diff G1024 S7 O8 P1 1000000vis", 1024, 7, 8, 1, 64, 4000.0, 497, 1, seed, limit=1_000_000)


def cored_quad_pol(seed: int = 0) -> Workload:
    """G=2048, S=7, O=8, P=4; 48 antennas in a 300 m core plus 16 out to 8 km; 2016 bl x 1024 t x 4 ch.

    The short core baselines put runs of adjacent samples on one oversampled-grid point, so compression
    (merging such runs) removes about 44% of the 8,257,536 records.
    """
    return observation("cored-quad-pol G2048 S7 O8 P4 8257536vis", 2048, 7, 8, 4, 64, 8000.0, 1024, 4, seed,
                       layout=lambda rng: cored_layout(48, 300.0, 16, 8000.0, rng))


def scaled_down(w: Workload, n: int) -> Workload:
    """The first n visibilities of a workload (same grid and kernel)."""
    return Workload(w.name + f" first{n}", w.G, w.S, w.oversample, w.npol, np.ascontiguousarray(w.uv[:n]),
                    np.ascontiguousarray(w.vis[:n]), np.ascontiguousarray(w.weights[:n]), w.beta, dict(w.meta))


def batched_counts(n_chan: int = 64, n_plane: int = 8, total: float = 20e6, lo: float = 1e3, hi: float = 1e6,
                   seed: int = 0) -> np.ndarray:
    """Visibility counts per (channel, plane), log-uniform on [lo, hi), rescaled to sum to about ``total``.

    Shape [n_chan, n_plane], int64, each at least 1.
    """
    rng = np.random.default_rng(seed)
    c = np.exp(rng.uniform(np.log(lo), np.log(hi), size=(n_chan, n_plane)))
    c = np.maximum(1, np.rint(c * (total / c.sum()))).astype(np.int64)
    return c


BATCH_PLANE_S = (7, 7, 9, 9, 11, 11, 15, 15)


def batched(seed: int = 0, n_chan: int = 64, n_plane: int = 8, total: float = 20e6, G: int = 1024,
            n_ant: int = 128, n_times: int = 128) -> list[list[Workload]]:
    """Channels x w-planes of single-pol G=1024 grids with uneven counts.

    S is (7, 7, 9, 9, 11, 11, 15, 15) by plane. Each (channel, plane) takes the
    first n samples of that channel's baseline-ordered track (8128 bl x 128 t
    for 128 antennas). Values are independent per (channel, plane).
    """
    counts = batched_counts(n_chan, n_plane, total, seed=seed)
    rng = np.random.default_rng(seed + 1)
    enu = antenna_layout(n_ant, 8000.0, rng)
    base = uv_tracks_m(enu, n_times, 1)[:, :, 0, :].reshape(-1, 2)
    out = []
    for k in range(n_chan):
        row = []
        for pl in range(n_plane):
            S = BATCH_PLANE_S[pl % len(BATCH_PLANE_S)]
            n = int(min(counts[k, pl], base.shape[0]))
            uv_m = base * (1.0 + CHANNEL_STEP * k)
            h = (S - 1) // 2
            uv = (uv_m[:n] * (0.9 * (G / 2 - h - 1) / float(np.max(np.abs(base * (1.0 + CHANNEL_STEP * (n_chan - 1))))))
                  ).astype(np.float64)
            vis = gaussian_values(rng, n, 1)
            row.append(Workload(f"batch ch{k} plane{pl}", G, S, 8, 1, np.ascontiguousarray(uv), vis,
                                np.ones(n, np.float32), beta=2.34 * S, meta=dict(channel=k, plane=pl)))
        out.append(row)
    return out


def random_uniform(G: int, S: int, oversample: int, npol: int, n: int, seed: int = 0, margin: float = 0.0) -> Workload:
    """Unordered uniform positions over the valid region (a worst case for coherence)."""
    rng = np.random.default_rng(seed)
    h = (S - 1) // 2
    lim = G / 2 - h - 1 - margin
    uv = rng.uniform(-lim, lim, size=(n, 2))
    return Workload(f"random G{G} S{S} O{oversample} P{npol} {n}vis", G, S, oversample, npol, uv,
                    gaussian_values(rng, n, npol), np.ones(n, np.float32), beta=2.34 * S)


def gaussian_sources_image(G: int, n_src: int = 5, seed: int = 0) -> np.ndarray:
    """Target image for the differentiation workload: n_src Gaussian sources, sigma 1..3 px,
    amplitude U(0.5, 1), centres in the central half of the image. [G, G] float64."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:G, 0:G].astype(np.float64)
    img = np.zeros((G, G))
    for _ in range(n_src):
        cx, cy = rng.uniform(G / 4, 3 * G / 4, size=2)
        sig = rng.uniform(1.0, 3.0)
        amp = rng.uniform(0.5, 1.0)
        img += amp * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * sig * sig))
    return img
