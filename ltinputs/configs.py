"""Workload presets: procedural box-room scenes sized like the paper's workloads.

The paper's own scenes (Bedroom, Tearoom, Museum; Table 1) are not available, so
seeded procedural scenes stand in for them.  Each preset fixes the scene recipe
(image size, VPL count, occluder boxes, materials) and the method's parameters
(slice count, sampling rate, rank, iteration count, cut bound).  Parameters are
plain numbers: no arithmetic of the method lives here.
"""
from __future__ import annotations

import copy

# Common method parameters (readings of the paper; Sec. 3-5):
#   eps_cut   lightcuts relative error bound for the conservative global cut (Sec. 3 item 1)
#   max_cut   cap on the global cut size (the paper's cuts hold ~800-900 nodes)
#   tau       coarsening threshold relative to the slice's estimated mean pixel (Eq. 2)
#   target_cut  > 0: coarsen each slice to this many nodes by cost order instead (Sec. 4)
#   rate      sampling rate rho = |Omega_s| / (m'_s n'_s)  (Sec. 5)
#   rank      completion rank r (the paper's q, Sec. 5)
#   als_iters fixed number of alternating least-squares sweeps
#   lam_rel   ridge term relative to the mean Gram diagonal
#   slice_bounds  (lo, hi): k-means slices held between lo and hi rows (small ones
#             merged into the nearest, large ones split by the 6-D median split)
#   slicing   "kmeans" (n_slices clusters) or "split6d" (the paper's recursive 6-D
#             binary split into slices of at most slice_size pixels)
#   n_meshes  icosphere occluders (triangles, mesh_subdiv subdivisions) besides the boxes
#   completion  "als" (masked ALS) or "adm" (the nonnegative ADM of App. A) with
#             adm_iters iterations, penalties adm_alpha_rel times the start's mean
#             Gram diagonal, and step gamma adm_gamma
_BASE = dict(
    target_cut=0,
    slicing="kmeans",
    slice_size=800,
    completion="als",
    adm_iters=100,
    adm_alpha_rel=0.3,
    adm_gamma=1.0,
    light_power=1.0,
    light_size=0.2,
    eps_cut=0.05,
    tau=0.02,
    lam_rel=1e-2,
    d_min=0.01,
    slice_feature_normal_weight=0.3,
    kmeans_iters=10,
    frame_seed=7,
)

CONFIGS = {
    # 64x64 points, 1024 VPLs, two floor boxes: the oracle renders it in seconds.
    "room64_vpl1k_2box": dict(
        _BASE, width=64, height=64, n_vpl=1024, n_big_boxes=2, n_small_boxes=0,
        glossy_frac=0.0, n_slices=16, rate=0.10, rate1=0.03, rank=8, als_iters=10,
        max_cut=1024, scene_seed=1001,
    ),
    # 256x256 points, 16384 VPLs, 200 random boxes behind a uniform grid.
    "room256_vpl16k_200box": dict(
        _BASE, width=256, height=256, n_vpl=16384, n_big_boxes=0, n_small_boxes=200,
        glossy_frac=0.0, n_slices=64, rate=0.05, rate1=0.015, rank=16, als_iters=10,
        max_cut=4096, scene_seed=1002,
    ),
    # 512x512 points, 65536 VPLs, 1000 boxes, Phong lobe on 30% of faces; uneven
    # k-means slices held between 128 and 4096 rows.
    "room512_vpl64k_1000box_glossy": dict(
        _BASE, width=512, height=512, n_vpl=65536, n_big_boxes=0, n_small_boxes=1000,
        glossy_frac=0.3, n_slices=128, slice_bounds=(128, 4096), rate=0.05, rate1=0.015, rank=16, als_iters=10,
        max_cut=2000, scene_seed=1003,
    ),
}


def get_config(name: str, **overrides) -> dict:
    """Return a copy of preset ``name`` with ``overrides`` applied."""
    if name not in CONFIGS:
        raise KeyError(f"unknown workload {name!r}; known: {sorted(CONFIGS)}")
    cfg = copy.deepcopy(CONFIGS[name])
    cfg.update(overrides)
    cfg["name"] = name
    return cfg


# 256x256 points, 16384 VPLs, the two-box generator of the tiny preset at full size:
# the scene family the learned-proposal experiments use (held-out seeds 5000-5019).
CONFIGS["room256_vpl16k_2box"] = dict(
    _BASE, width=256, height=256, n_vpl=16384, n_big_boxes=2, n_small_boxes=0,
    glossy_frac=0.0, n_slices=64, rate=0.15, rate1=0.002, rank=16, als_iters=10,
    max_cut=16384, tau=0.0005, d_min=0.1, scene_seed=5000,
)

# 256x256 points, 16384 VPLs, two boxes, colour: RGB face albedos and a warm light
# (the paper's coloured scenes); the three channels are stacked as rows of a slice.
CONFIGS["room256_vpl16k_2box_rgb"] = dict(
    CONFIGS["room256_vpl16k_2box"], rgb=True, light_rgb=(1.0, 0.85, 0.7),
)

# Triangle-mesh occluders: icospheres (320 triangles each) on the floor besides the
# two boxes; the tiny form for the oracle, the full form at the bench size.
CONFIGS["room64_vpl1k_mesh"] = dict(
    CONFIGS["room64_vpl1k_2box"], n_meshes=2, mesh_subdiv=2, scene_seed=1004,
)
CONFIGS["room256_vpl16k_mesh"] = dict(
    CONFIGS["room256_vpl16k_2box"], n_meshes=6, mesh_subdiv=3, scene_seed=5001,
)

# 1024x1024 points, 262144 VPLs, 2000 boxes with a Phong lobe on 30% of faces,
# 256 k-means slices, rank up to 32 chosen per slice (the large combined workload,
# sized like the paper's Tearoom: 786K pixels, 231K VPLs).
CONFIGS["room1024_vpl256k_2000box_glossy"] = dict(
    _BASE, width=1024, height=1024, n_vpl=262144, n_big_boxes=0, n_small_boxes=2000,
    glossy_frac=0.3, n_slices=256, rate=0.05, rate1=0.002, rank=32, rank_cols=512, als_iters=10,
    max_cut=16384, tau=0.0005, scene_seed=1005,
)
