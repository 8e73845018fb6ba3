"""Compass tuning constants (inputs to both the oracle and the GPU path).

The paper names its two algorithm parameters, the number of sectors searched
(1, 3 or 5) and the number of valid candidates tested (1..16), Sec. V and
Sec. VI-B, and keeps (5 sectors, 8 candidates) as its trade-off (Sec. VII).
It gives no value for any tolerance, so the others are this project's
choices for the synthetic detector:

* qop_max: 1/1.5 GeV^-1, the smallest momentum the generator makes.
* window half-width in layer l: kick_k*qop_max*|z_l - z_kink| + tol_win.
* pair cuts: residual slope within kick_k*qop_max + tol_slope; the pair
  line's residual at the kink plane within tol_kink.
* collection: nearest hit within tol_col of the pair line.
* fit: hit sigma = pitch/sqrt(12), VELO priors sigma_x, sigma_tx.
* gec_max_hits: the Global Event Cut applied before the tracking (Sec. VI):
  events with more UT hits are not searched; 0 = no cut.  The paper takes
  LHCb's cut and gives no value.
* output_order: 0 = each VELO track's result in its own slot; 1 = the
  paper's output order (found tracks of an event at indices taken from an
  atomic counter, Sec. V-B).  Not an input of the method's arithmetic.
"""
from __future__ import annotations

import dataclasses
import math


@dataclasses.dataclass
class CompassParams:
    n_sectors: int = 5
    n_candidates: int = 8
    qop_max: float = 1.0 / 1.5
    tol_win: float = 1.0
    tol_kink: float = 0.5
    tol_col: float = 0.4
    tol_slope: float = 0.01
    chi2ndof_max: float = 25.0
    sigma_hit: float = 0.187 / math.sqrt(12.0)
    sigma_x_prior: float = 0.01
    sigma_tx_prior: float = 1e-5
    z_kink: float = 2500.0
    kick_k: float = 1.2
    gec_max_hits: int = 0
    output_order: int = 0

    def replace(self, **kw) -> "CompassParams":
        return dataclasses.replace(self, **kw)
