"""Seeded synthetic phantoms shaped like the paper's 2-D Ra-223 SPECT study.

The paper (Sec. "Synthetic phantom model") images an elliptical body with
semi-axes 11 cm x 9 cm that holds circular lesions, and a water-based
attenuation map whose density varies between regions.  These helpers build
the same kind of object on the pixel grid of a workload: a relative-density
map ``rho`` (water = 1, bone = 1.6, air = 0) and a true activity map.

Rasterisation is by pixel-centre sampling: a pixel takes the value of the
shape that contains its centre.  Pixel (ix, iy) has its centre at
``((ix + 0.5 - n/2) h, (iy + 0.5 - n/2) h)`` cm and is stored at ``iy*n + ix``.

This module is input generation only.  It holds none of the reconstruction
arithmetic and is shared, as inputs, by the oracle tests and the CUDA path.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

ELLIPSE_SEMI_AXES_CM = (11.0, 9.0)
BONE_DENSITY = 1.6
LESION_TO_BACKGROUND = 8.0


@dataclass(frozen=True)
class Disc:
    x_cm: float
    y_cm: float
    r_cm: float


@dataclass(frozen=True)
class PhantomSpec:
    """Ellipse body + optional bone disc + circular lesions (all centred in cm).

    ``rim_cm`` > 0 gives the body a denser outer rim (the paper's attenuation
    map has a rim of 0.21 and an inner region of 0.18 1/cm at 85 keV, i.e.
    water whose density differs between the two)."""

    bone: Disc | None
    lesions: tuple[Disc, ...]
    semi_axes_cm: tuple[float, float] = ELLIPSE_SEMI_AXES_CM
    lesion_ratio: float = LESION_TO_BACKGROUND
    rim_cm: float = 0.0
    rim_density: float = 1.0


# Two lesions and a bone disc (the 32x32 and 64x64 workloads).
TWO_LESION = PhantomSpec(
    bone=Disc(-5.0, 0.0, 2.0),
    lesions=(Disc(4.0, 3.0, 1.4), Disc(4.0, -3.0, 1.0)),
)


def _four_lesions() -> tuple[Disc, ...]:
    out = []
    for r_cm, deg in zip((1.0, 2.0, 3.0, 4.0), (45.0, 135.0, 225.0, 315.0)):
        t = np.deg2rad(deg)
        out.append(Disc(5.5 * float(np.cos(t)), 5.5 * float(np.sin(t)), r_cm))
    return tuple(out)


# Four lesions of radius 1-4 cm (the 128x128 workloads).
FOUR_LESION = PhantomSpec(bone=Disc(0.0, 0.0, 1.2), lesions=_four_lesions())


def paper_study_phantom(sbr: float = 4.0) -> PhantomSpec:
    """The paper's study object: four lesions of radius 7/10/12/14 mm placed
    symmetrically about the centre, signal-to-background ratio ``sbr``, and a
    rim/inner attenuation map (0.21 vs 0.18 1/cm at 85 keV)."""
    lesions = []
    for r_cm, deg in zip((0.7, 1.0, 1.2, 1.4), (45.0, 135.0, 225.0, 315.0)):
        t = np.deg2rad(deg)
        lesions.append(Disc(4.5 * float(np.cos(t)), 4.5 * float(np.sin(t)), r_cm))
    return PhantomSpec(bone=None, lesions=tuple(lesions), lesion_ratio=sbr, rim_cm=1.0,
                       rim_density=0.21 / 0.18)


def random_water_bone_object(seed: int, k: int) -> PhantomSpec:
    """Object ``k`` of a seeded family of random water/bone ellipses (the
    surrogate's training objects): semi-axes 7-12.5 cm x 5.5-10 cm, a denser
    rim in half of them, a bone disc of radius 0.8-2.5 cm somewhere inside,
    and two to four lesions at 2:1-8:1."""
    rng = np.random.Generator(np.random.Philox(key=[seed, k]))
    ax, ay = rng.uniform(7.0, 12.5), rng.uniform(5.5, 10.0)

    def inside(margin):
        while True:
            x, y = rng.uniform(-ax, ax), rng.uniform(-ay, ay)
            if (x / (ax - margin)) ** 2 + (y / (ay - margin)) ** 2 <= 1.0:
                return float(x), float(y)

    rb = rng.uniform(0.8, 2.5)
    bx, by = inside(rb + 0.5)
    lesions = []
    for _ in range(int(rng.integers(2, 5))):
        r = rng.uniform(0.6, 2.0)
        lx, ly = inside(r + 0.3)
        lesions.append(Disc(lx, ly, float(r)))
    rim = float(rng.uniform(0.5, 1.5)) if rng.random() < 0.5 else 0.0
    return PhantomSpec(bone=Disc(bx, by, float(rb)), lesions=tuple(lesions),
                       semi_axes_cm=(float(ax), float(ay)),
                       lesion_ratio=float(rng.uniform(2.0, 8.0)), rim_cm=rim,
                       rim_density=float(rng.uniform(1.05, 1.2)))


def pixel_centres_cm(n: int, pixel_cm: float) -> tuple[np.ndarray, np.ndarray]:
    """Return (x, y) pixel-centre coordinates, each shaped (n, n) as [iy, ix]."""
    c = (np.arange(n, dtype=np.float64) + 0.5 - n / 2.0) * pixel_cm
    y, x = np.meshgrid(c, c, indexing="ij")
    return x, y


def _inside(x, y, d: Disc):
    return (x - d.x_cm) ** 2 + (y - d.y_cm) ** 2 <= d.r_cm ** 2


@dataclass
class Phantom:
    rho: np.ndarray          # (n, n) float32 relative density
    activity: np.ndarray     # (n, n) float32 true activity (background 1)
    lesion_masks: list = field(default_factory=list)  # per lesion (n, n) bool


def make_phantom(spec: PhantomSpec, n: int, pixel_cm: float) -> Phantom:
    x, y = pixel_centres_cm(n, pixel_cm)
    ax, ay = spec.semi_axes_cm
    body = (x / ax) ** 2 + (y / ay) ** 2 <= 1.0
    rho = np.where(body, 1.0, 0.0)
    if spec.rim_cm > 0:
        inner = (x / (ax - spec.rim_cm)) ** 2 + (y / (ay - spec.rim_cm)) ** 2 <= 1.0
        rho = np.where(body & ~inner, spec.rim_density, rho)
    if spec.bone is not None:
        bone = body & _inside(x, y, spec.bone)
        rho = np.where(bone, BONE_DENSITY, rho)
    act = np.where(body, 1.0, 0.0)
    masks = []
    for d in spec.lesions:
        m = body & _inside(x, y, d)
        masks.append(m)
        act = np.where(m, spec.lesion_ratio, act)
    return Phantom(rho.astype(np.float32), act.astype(np.float32), masks)
