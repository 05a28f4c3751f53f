"""CPU oracle for the AFC hot path (test infrastructure; see afc_oracle)."""
from .afc_oracle import *  # noqa: F401,F403
