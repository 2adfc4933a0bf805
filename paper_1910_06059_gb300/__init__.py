"""GB300-native fully-implicit black-oil Newton step (arXiv 1910.06059).

The compute path is ``libbo.so`` (hand-written CUDA for sm_103a behind the C
ABI of ``include/bo.h``); this package only marshals arguments to it.
"""
from ._lib import BoError, EXPORTED, LIB_PATH, load, newton_opts  # noqa: F401
from .sim import Sim  # noqa: F401
from .ensemble import Ensemble  # noqa: F401
from .report import StepLog  # noqa: F401


def build(force: bool = False) -> str:
    """Compile libbo.so in-tree for sm_103a."""
    from .build import build as _build
    return _build(force=force)
