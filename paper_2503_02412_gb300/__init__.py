"""GB300-native SE(2)-grid traversability assessment (SEB-Naver, arXiv 2503.02412, Sec. V).

The compute path is libseb.so (hand-written CUDA for sm_103a behind a C ABI, include/seb.h);
this package only marshals torch tensors and streams into it.
"""
from . import abi  # noqa: F401
from .elevation import ElevationMap, scan_pose  # noqa: F401
from .inpaint import inpaint_nearest  # noqa: F401
from .lookup import SE2Grid, SE2Lookup, risk_sdf, se2_lookup  # noqa: F401
from .maps import CHANNELS, SebMap, SebParams, encode_bf16_tiled, tiled_parts, tiled_window  # noqa: F401

__all__ = ["abi", "SebMap", "SebParams", "CHANNELS", "encode_bf16_tiled", "tiled_parts", "tiled_window", "SE2Grid", "SE2Lookup", "se2_lookup", "risk_sdf", "inpaint_nearest", "ElevationMap", "scan_pose"]
