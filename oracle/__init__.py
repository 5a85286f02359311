"""CPU float64 oracle (test infrastructure only; see conreg_oracle)."""
from .conreg_oracle import Oracle, GreedyResult, cg, cholesky_solve  # noqa: F401
