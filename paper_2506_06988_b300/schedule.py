"""Host-side schedule of the joint optimisation (Sec. 3.4, Sec. 4.1,
Algorithm 1).

The texture loss is off during a warm-up in which the hybrid render alone is
supervised with the photometric loss (N = 3k iterations), on with weight
lambda = 0.1 strictly between the warm-up and the end of the 3DGS
densification (15k iterations), and off afterwards.  Iterations count from 0
as in Algorithm 1, whose test is i > i_warm-up and i < i_densification.
"""
from __future__ import annotations

__all__ = ["texture_loss_weight"]

WARMUP = 3000
DENSIFY_UNTIL = 15000
LAMBDA_T = 0.1


def texture_loss_weight(iteration: int, lam: float = LAMBDA_T, warmup: int = WARMUP,
                        until: int = DENSIFY_UNTIL) -> float:
    """lambda_t of the joint loss at training iteration ``iteration``."""
    return float(lam) if warmup < iteration < until else 0.0
