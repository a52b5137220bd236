"""GB300 isochrone queries (Baum et al., "Fast Computation of Isochrones in Road
Networks"): host contraction hierarchy + CUDA PHAST sweep for sm_103a, behind
the C ABI in include/iso.h.  The Python names mirror the C entry points."""

from ._lib import (  # noqa: F401
    CH, DeviceGraph, IsoError, Workspace, iso_build_ch, iso_load_ch, iso_query, iso_upload_graph, lib,
    INF, ISO_OK, ISO_E_INVAL, ISO_E_NOMEM, ISO_E_OVERFLOW, ISO_E_CUDA, ISO_E_TIMEOUT, ISO_E_IO, ISO_E_NODEV,
)

__all__ = ["CH", "DeviceGraph", "Workspace", "IsoError", "iso_build_ch", "iso_load_ch", "iso_upload_graph",
           "iso_query", "lib"]
