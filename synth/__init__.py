"""Seeded synthetic digital-holography streams (inputs only; no EM arithmetic)."""
from .ddh_synth import (  # noqa: F401
    StreamConfig, config_single_64, config_single_256, config_batched, config_adjoint,
    config_service, velocity_magnitude, paper_velocity, make_stream, Stream,
)
