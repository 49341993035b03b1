"""Seeded synthetic inputs (RF phantoms and workload recipes); no beamforming arithmetic."""
from . import configs, phantom  # noqa: F401
