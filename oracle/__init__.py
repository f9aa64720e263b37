"""FP64 CPU oracle of the four Tucker methods.  Test infrastructure only: the test suite, the
smoke check and the benchmark's CPU-baseline leg use it; the GPU library never does."""
from . import tucker_oracle  # noqa: F401
