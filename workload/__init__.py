"""Seeded synthetic LQ workloads shaped like the Kuka IIWA-14 tracking problems.

This package only draws random numbers and lays them out; it contains none of
the solver's arithmetic.  Both the CUDA path and the CPU oracle take their
inputs from here.
"""
from .gen import (  # noqa: F401
    LQ, LQBatch, kuka_lq, kuka_batch, concat_batch, batch_horizons,
    warm_noise, warm_start, loss_weights, to_f32,
    CONFIG_SMALL, CONFIG_SWEEP, CONFIG_BATCH, CONFIG_GRAD, CONFIG_LARGE,
)
