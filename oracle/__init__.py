"""FP64 CPU oracle (test infrastructure only; see ``spec_oracle``)."""
from .spec_oracle import *  # noqa: F401,F403
