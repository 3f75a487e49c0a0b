"""Seeded synthetic detector events shared by the CUDA path, the oracle and the bench.

This package simulates the detector: particles on exact helices in a uniform
solenoid field, their crossings with barrel cylinders and endcap disks, Gaussian
hit smearing, hit inefficiency and uniform noise.  It contains none of the
Kalman-filter method (no propagation-to-surface solver, no Jacobian, no update):
particles start on the beam line, where the crossing of a cylinder has a closed
form; neither implementation of the method uses it (both solve crossings from
arbitrary points on the track).

The paper ("Parallelized and Vectorized Tracking Using Kalman Filters with CMS
Detector Geometry and Events", sec. 2.1-2.2 and 3) runs on CMSSW ttbar + PU70
events with the CMS-2017 geometry; neither is available, so the configurations in
`configs.py` stand in for them (synthetic, seeded, with the geometry, field,
resolutions, occupancy and pT/eta spectra described there).
"""
from .configs import CONFIGS, K_FIELD, get_config, layer_table
from .events import Batch, make_batch, make_event

__all__ = ["CONFIGS", "K_FIELD", "get_config", "layer_table", "Batch", "make_batch", "make_event"]
