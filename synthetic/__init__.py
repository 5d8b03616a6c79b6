"""Seeded synthetic inputs (phantoms, scanner presets, Monte-Carlo events).

Input generation only: nothing here evaluates the reconstruction model.  Both
the FP64 oracle tests and the CUDA path draw their inputs from this package.
"""
from .phantom import (FOUR_LESION, TWO_LESION, Phantom, PhantomSpec, make_phantom,
                      pixel_centres_cm, random_water_bone_object)
from .presets import PRESETS, Scenario, preset
from .mc import EventList, simulate, simulate_cached

__all__ = ["FOUR_LESION", "TWO_LESION", "Phantom", "PhantomSpec", "make_phantom",
           "random_water_bone_object",
           "pixel_centres_cm", "PRESETS", "Scenario", "preset", "EventList", "simulate",
           "simulate_cached"]
