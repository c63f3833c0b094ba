"""GB300 (sm_103a) library for the time step of the D2Q9 MRT pseudopotential
lattice Boltzmann model with fluid-solid interaction (Li, Luo, Kang & Chen,
"Contact angles in the pseudopotential lattice Boltzmann modeling of
wetting").  The C ABI is include/lbm.h; this package is its Python face."""
from ._lib import LbmError, load  # noqa: F401
from .lattice import Lattice, default_params  # noqa: F401
