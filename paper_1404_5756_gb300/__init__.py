"""GB300 recursive-filter horizontal covariance operator V_H (3rd-RF and
1st-RF x K) behind the C ABI of include/rfvh.h."""
from ._lib import RF_NORM_GAUSS_PEAK, RF_NORM_UNIT_SUM, RFError  # noqa: F401
from .vh import Graph, Options, Plan, VhFunction, vh  # noqa: F401
