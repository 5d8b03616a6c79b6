"""Named synthetic workloads.

Each preset fixes the grid, the scanner, the spectrum, the energy model, the
phantom, the event count and the seed.  The 2-D SPECT study of the paper
(Sec. "SPECT simulation") is the model: parallel-hole collimator whose blur
grows with depth, a NaI detector with 10% FWHM at 140 keV that scales as
1/sqrt(E), three emission lines of Ra-223 (82/154/270 keV with yields
0.6/0.2/0.2) and a water attenuation curve that is linear between knots.

``small_*`` presets are extra parity cases sized so that the FP64 oracle
finishes in seconds.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

from .phantom import (FOUR_LESION, TWO_LESION, Phantom, PhantomSpec, make_phantom,
                      paper_study_phantom)


@dataclass(frozen=True)
class Scenario:
    name: str
    n: int
    pixel_cm: float
    n_angles: int
    n_bins: int
    scatter_n: int
    n_events: int
    seed: int
    n_subsets: int
    n_iters: int
    phantom: PhantomSpec = TWO_LESION
    bin_cm: float = 0.0            # 0 -> n * pixel_cm / n_bins (detector spans the image)
    r_det_cm: float = 0.0          # 0 -> n * pixel_cm / 2
    coll_fwhm0_cm: float = 0.3
    coll_fwhm_slope: float = 0.02
    scan_time: float = 1.0
    knot_keV: tuple = (82.0, 154.0, 270.0)
    mu_water_cm: tuple = (0.184, 0.148, 0.121)
    line_keV: tuple = (82.0, 154.0, 270.0)
    yields: tuple = (0.6, 0.2, 0.2)
    fwhm_frac: float = 0.10
    e_ref_keV: float = 140.0
    fwhm_exponent: float = -0.5
    windows: tuple = ((50.0, 300.0),)

    @property
    def length_cm(self) -> float:
        return self.n * self.pixel_cm

    @property
    def bin_width_cm(self) -> float:
        return self.bin_cm if self.bin_cm > 0 else self.length_cm / self.n_bins

    @property
    def detector_radius_cm(self) -> float:
        return self.r_det_cm if self.r_det_cm > 0 else self.length_cm / 2.0

    def make_phantom(self) -> Phantom:
        return make_phantom(self.phantom, self.n, self.pixel_cm)

    def with_(self, **kw) -> "Scenario":
        return replace(self, **kw)


PRESETS: dict[str, Scenario] = {
    # 32x32, 0.8 cm, 32 angles, 32 bins, 16x16 scatter grid, 2000 events, 4x1.
    "lmmew_32": Scenario("lmmew_32", 32, 0.8, 32, 32, 16, 2000, 0, 4, 1),
    # 64x64, 0.6 cm, 60 angles, 64 bins, 64x64 scatter grid, 300k events, 8x10.
    "lmmew_64": Scenario("lmmew_64", 64, 0.6, 60, 64, 64, 300_000, 1, 8, 10),
    # 128x128, 0.3 cm, 120 angles, 128 bins, 64x64 scatter, 1M events, 8x10.
    "lmmew_128": Scenario("lmmew_128", 128, 0.3, 120, 128, 64, 1_000_000, 2, 8, 10,
                          phantom=FOUR_LESION),
    # 128x128 at 2M events (the learned-surrogate evaluation size).
    "lmmew_128_2m": Scenario("lmmew_128_2m", 128, 0.3, 120, 128, 64, 2_000_000, 4, 8, 10,
                             phantom=FOUR_LESION),
    # Oracle-sized parity cases: several kernel tiles plus ragged tails.
    "small_16": Scenario("small_16", 16, 1.6, 12, 20, 8, 700, 11, 3, 2),
    "small_24": Scenario("small_24", 24, 1.2, 10, 24, 24, 900, 12, 2, 2),
    "small_32_4w": Scenario("small_32_4w", 32, 0.8, 16, 40, 16, 1500, 13, 4, 1,
                            windows=((68.0, 102.0), (123.0, 184.0), (243.0, 297.0))),
    "tiny_8": Scenario("tiny_8", 8, 3.2, 4, 10, 4, 64, 14, 2, 2),
    # The paper's comparison study (Sec. Experiments): 64x64 grid of 4.6 mm,
    # 120 angles, the three photopeak windows, ~1e4 events per realisation,
    # 4 subsets x 16 iterations, four lesions at 4:1.
    "paper_study": Scenario("paper_study", 64, 0.46, 120, 64, 32, 10_000, 21, 4, 16,
                            phantom=paper_study_phantom(4.0),
                            windows=((68.0, 102.0), (123.0, 184.0), (243.0, 297.0))),
    "noscatter_16": Scenario("noscatter_16", 16, 1.6, 8, 16, 0, 400, 15, 2, 3),
}


def preset(name: str) -> Scenario:
    return PRESETS[name]
