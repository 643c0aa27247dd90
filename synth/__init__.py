"""Seeded synthetic inputs (meshes, strokes, cameras, lassos) shared by the tests, the
benchmark and the oracle checks.  This package holds no step of the layer-editing
method itself: it only produces plain arrays."""
from .mesh import (Mesh, displaced_sphere, grid_patch, random_soup, torus, uv_square_patch, vessel_charts,
                   vessel_cylindrical)
from .noise import GradientNoise3
from .workload import (BatchModel, Camera, Lasso, Strokes, Workload, batch_model, config_batch, bbox_diag, config_large, config_roofline,
                       config_small, lassos, look_at, orbit_camera, orthographic01, perspective01,
                       project_px, sphere_strokes, star_lasso, surface_points)
