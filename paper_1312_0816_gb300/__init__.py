"""GB300-native vector navigator: distance to the next boundary, Contains and
Safety for baskets of tracks inside one mother volume (Box, Tube, Cone, tube
segment and polycone daughters), after "Vectorising the detector geometry to
optimize particle transport".  The compute path is libgeonav.so (hand-written CUDA for sm_103a)
behind the C ABI of include/geo.h; `geonav` is its Python binding."""
from .geonav import (GEO_BOX, GEO_CONE, GEO_FP32_REFINE, GEO_FP64, GEO_PCON, GEO_SAFETY_ESTIMATE, GEO_TUBE,  # noqa: F401
                     GEO_TUBS, GEO_MAX_PLANES, GEO_TILE_TRACKS, GeoError, Volume,
                     geo_build_volume, geo_contains, geo_destroy_volume, geo_dist_to_boundary,
                     geo_dist_to_boundary_host, geo_dist_to_boundary_stats, geo_check_device_status, geo_probe_pipe,
                     geo_safety, geo_status_string, geo_volume_info, load, Batch, geo_build_batch,
                     geo_destroy_batch, geo_dist_to_boundary_batched, geo_dist_to_boundary_batched_noalloc,
                     geo_adjoint_workspace_size, geo_dist_to_boundary_adjoint,
                     geo_shape_query, GEO_Q_DIST_OUT, GEO_Q_DIST_IN, GEO_Q_SAFETY_OUT, GEO_Q_SAFETY_IN,
                     GEO_Q_CONTAINS, World, geo_build_world, geo_destroy_world, geo_world_info,
                     geo_world_nodes, geo_world_locate, geo_world_step, geo_selftest_wait_timeout,
                     geo_debug_fail_alloc)
