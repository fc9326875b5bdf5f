"""WaveHoltz on overset grids for one GB300 GPU (sm_103a).

* :mod:`paper_2504_03074_gb300.grids` -- seeded overset grid descriptions and sources;
* :mod:`paper_2504_03074_gb300.waveholtz` -- the binding to ``libwaveholtz`` (C ABI in
  ``include/waveholtz.h``), loaded on first use; it raises if the CUDA library is
  missing: there is no CPU fallback.
"""
__all__ = ["grids", "waveholtz"]
