"""FP64 CPU oracle of the digital shearlet transform (test infrastructure only)."""
from .shearlet_oracle import *  # noqa: F401,F403
