"""GB300-native ensemble DNS hot path (Bentkamp & Wilczek's ensemble method).

``libens.so`` (CUDA, sm_103a; C ABI in ``include/ens.h``) advances a
heterogeneous ensemble of forced periodic-box Navier-Stokes members, reduces
each member's velocity-gradient tensor to Q-R, dissipation and enstrophy
histograms plus moments, and mixes them over lambda.  :mod:`.ens` is the thin
Python binding.
"""
from .ens import Ensemble, Member, hist_spec  # noqa: F401
