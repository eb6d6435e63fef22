"""CPU oracle (test infrastructure only; see pint_oracle's docstring)."""
from .pint_oracle import *  # noqa: F401,F403
