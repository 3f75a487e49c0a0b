"""Algorithmic work per unit of the finding and fitting kernels (frozen counts).

Counted by hand from the formulation in csrc/mkf_math.cuh, one FMA = 2 flops,
one add / multiply / compare-select = 1 flop, each SFU-class call (sin, cos,
sqrt, reciprocal, division, atan2) = 1 flop.  The counts are the minimal work of
the formulation (symmetric-packed covariance, structured Jacobian, float pairs
for position and phi), not what a particular kernel happens to execute.

Candidate-layer (one parent propagated to one layer and searched):
  path to the next surface (cylinder quadratic with exact R^2 - r^2,
  about 1.2 surfaces tried per step)            ~ 110
  extent check at the crossing                  ~  30
  propagation + Jacobian (J = A + d g^T)        ~  90
  transport C' = J C J^T, structured           ~ 310
  float-pair position and phi moves             ~  40
  frame, H C, S, S^-1                           ~  70
  chi2 window and bin range                     ~  50
                                                  ----
                                                  700
Hit tested inside the window rectangle: difference vector, cross and dot
products, atan2, (u, v), chi2 = r^T S^-1 r        45
Kalman update of a kept child: frame, H C, S^-1, residual, chi2, gain K (6x2),
state update with float pairs, C -= K (H C) on 21 entries     300
Fit, per track-layer: path + propagation + transport + update   850
"""

FLOPS_PER_CAND_LAYER = 700
FLOPS_PER_HIT_TESTED = 45
FLOPS_PER_UPDATE = 300
FLOPS_PER_FIT_LAYER = 850

# Bytes a finding step must move at least: every hit read once (16-byte binned
# record), seeds (12 B), outputs per seed (27 floats + chi2 + n_hits + status +
# hit list of max_out int32).
BYTES_PER_HIT = 16


def find_flops(cand_layers: int, hits_tested: int, updates: int) -> int:
    return (FLOPS_PER_CAND_LAYER * int(cand_layers) + FLOPS_PER_HIT_TESTED * int(hits_tested)
            + FLOPS_PER_UPDATE * int(updates))


def fp32_peak_tflops(sm_count: int, sm_mhz: float) -> float:
    """FP32 FMA-pipe peak: 128 FP32 lanes per SM, 2 flops per FMA."""
    return sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12
