"""GB300-native locally relaxed entropy-stable RK step (Ranocha, Dalcin & Parsani 2020).

The compute path is the CUDA library ``libes.so`` (C ABI in ``include/es.h``);
``_binding`` marshals torch tensors / numpy arrays to it, ``solver`` is a small
convenience layer, ``inputs`` builds the synthetic initial states.
"""
from . import _binding  # noqa: F401
from ._binding import (ES_BC_PERIODIC, ES_BC_STATE, ES_BC_VISCOUS_SHOCK, ES_FP64, ES_FP64X, ES_MIXED, ES_MIXED_FF, ES_RELAX_GLOBAL, ES_RELAX_LOCAL, ES_RELAX_NONE,  # noqa: F401
                       ES_RK_BS3, ES_RK_RK4, ES_RK_RK65, ESError, make_config)
