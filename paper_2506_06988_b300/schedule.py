"""Host-side schedule of the joint optimisation (Sec. 3.4, Sec. 4.1).

The texture loss is off during a warm-up in which the Gaussians alone are
fitted with the photometric loss (N = 3k iterations), on with weight
lambda = 0.1 until the 3DGS densification ends (15k iterations), and off
afterwards, when the hybrid render alone is supervised.
"""
from __future__ import annotations

__all__ = ["texture_loss_weight"]

WARMUP = 3000
DENSIFY_UNTIL = 15000
LAMBDA_T = 0.1


def texture_loss_weight(iteration: int, lam: float = LAMBDA_T, warmup: int = WARMUP,
                        until: int = DENSIFY_UNTIL) -> float:
    """lambda_t of the joint loss at a (0-based) training iteration."""
    return float(lam) if warmup <= iteration < until else 0.0
