"""Seeded synthetic inputs shared by the oracle and the CUDA path (no method arithmetic)."""
from .models import *  # noqa: F401,F403
from .models import CONFIGS, anisotropic, fluid_params, random_state, small_model, layered_model  # noqa: F401
