"""The oracle's pins catch planted mistakes (CPU; no GPU).

Each case plants one plausible mistake -- a dropped term, a wrong sign, index
or comparison, a transposed operand -- into a copy of the C oracle (walks,
gains, endpoint grid and reductions of Section III), builds that copy, and runs
the pins of test_oracle_pins.py against it: at least one pin must fail.  An
unmodified copy built the same way must pass them all.  The oracle itself is not
touched; the planted copies live in a temporary directory.  Every planted
mistake keeps memory accesses in bounds (walk indices stay clamped and checked,
buffers are written only below their capacity).
"""

import pytest

import oracle
import test_oracle_pins as pins
from oracle.build import SRC, compile_source

PINS = ([("test_hand_cases_all_walks", {}), ("test_hand_tie_cases", {}), ("test_tie_gap_by_hand", {}),
         ("test_segments_start_at_the_camera_in_voxel_units", {}), ("test_hand_case_eq2", {})]
        + [("test_walks_match_brute_force", {"dims": d}) for d in [(7, 5, 9), (16, 16, 16), (1, 12, 3)]]
        + [("test_f32_walk_differs_from_f64_only_at_ties", {}), ("test_walk_is_a_connected_monotone_path", {}),
           ("test_all_unknown_count_closed_form", {}), ("test_all_free_and_all_occupied", {}),
           ("test_all_occupied_eq2_gains_entry_voxel", {})]
        + [("test_axis_aligned_lengths", {"axis": a, "sign": s}) for a in range(3) for s in (1, -1)]
        + [("test_occlusion_wall_closed_form", {}), ("test_ray_stops_at_first_occupied", {})]
        + [("test_revealing_voxels_never_increases_ig", {"metric": m}) for m in ("count", "eq2", "entropy")]
        + [("test_view_ig_is_permutation_invariant_sum_of_rays", {}), ("test_traj_ig_is_sum_over_csr_ranges", {}),
           ("test_threads_do_not_change_results", {}), ("test_entropy_values", {}), ("test_gain_table", {}),
           ("test_long_sums_are_accumulated_in_fp64", {})]
        + [("test_endpoint_grid_geometry", {"grid_mode": g, "range_mode": r})
           for g in ("corners", "centers") for r in ("planar", "spherical")]
        + [("test_perspectives_nearer_the_poi_gain_less", {})])

F32, F64, BRUTE = "int64_t orc_walk_f32(", "int64_t orc_walk_f64(", "int64_t orc_walk_brute("

# (name, anchor, text, planted text): the first occurrence of text after anchor is replaced
MUTANTS = [
    ("tie_break_z_first", F32,
     "int a = (tn[0] <= tn[1] && tn[0] <= tn[2]) ? 0 : (tn[1] <= tn[2] ? 1 : 2);",
     "int a = (tn[0] < tn[1] && tn[0] < tn[2]) ? 0 : (tn[1] < tn[2] ? 1 : 2);"),
    ("first_crossing_plane_off_by_one", F32,
     "tn[a] = step[a] != 0 ? ((float)(idx[a] + (step[a] > 0)) - o[a]) * inv[a] : INFINITY;",
     "tn[a] = step[a] != 0 ? ((float)(idx[a]) - o[a]) * inv[a] : INFINITY;"),
    ("near_clip_dropped", F32, "tmin = lo > tmin ? lo : tmin;", "(void)lo;"),
    ("start_from_unclipped_origin", F32, "float p = o[a] + tmin * d[a];", "float p = o[a];"),
    ("end_test_inclusive", F32, "if (!(tn[a] < tmax)) break;", "if (!(tn[a] <= tmax)) break;"),
    ("next_plane_on_wrong_side", F32,
     "    tn[a] = ((float)(idx[a] + (step[a] > 0)) - o[a]) * inv[a];",
     "    tn[a] = ((float)(idx[a] + (step[a] < 0)) - o[a]) * inv[a];"),
    ("f64_crossing_always_upper_plane", F64,
     "tn[a] = step[a] != 0 ? ((double)(idx[a] + (step[a] > 0)) - o[a]) / d[a] : INFINITY;",
     "tn[a] = step[a] != 0 ? ((double)(idx[a] + 1) - o[a]) / d[a] : INFINITY;"),
    ("brute_counts_touching_voxels", BRUTE, "if (inside && tin < tout) {", "if (inside && tin <= tout) {"),
    ("brute_slab_bounds_unordered", BRUTE,
     "double lo = t0 < t1 ? t0 : t1, hi = t0 < t1 ? t1 : t0;", "double lo = t0, hi = t1;"),
    ("entropy_in_nats", "double orc_entropy(",
     "return -p * log2(p) - (1.0 - p) * log2(1.0 - p);", "return -p * log(p) - (1.0 - p) * log(1.0 - p);"),
    ("eq2_free_and_occupied_swapped", "void orc_voxel_gain(",
     "*g = occ ? 1.0 - (double)p : (fre ? (double)p : 1.0);",
     "*g = occ ? (double)p : (fre ? 1.0 - (double)p : 1.0);"),
    ("occupied_threshold_inclusive", "void orc_voxel_gain(",
     "int occ = p > prm->occ_threshold;", "int occ = p >= prm->occ_threshold;"),
    ("free_counted_as_unknown_on_state_maps", "void orc_voxel_gain(",
     "*g = s == 0 ? 1.0 : 0.0;", "*g = s <= 1 ? 1.0 : 0.0;"),
    ("free_counted_as_unknown_on_probability_maps", "void orc_voxel_gain(",
     "*g = (!occ && !fre) ? 1.0 : 0.0;", "*g = !occ ? 1.0 : 0.0;"),
    ("occluding_voxel_never_counted", "static int visit_gain(",
     "if (acc->prm->include_hit) acc->ig += g;", "(void)g;"),
    ("walk_continues_past_occupied", "static int visit_gain(",
     "    if (acc->prm->include_hit) acc->ig += g;\n    return 1;",
     "    if (acc->prm->include_hit) acc->ig += g;\n    return 0;"),
    ("voxel_index_transposed", "static int visit_gain(",
     "int64_t idx = ((int64_t)z * acc->m->ny + y) * acc->m->nx + x;",
     "int64_t idx = ((int64_t)x * acc->m->ny + y) * acc->m->nz + z;"),
    ("mean_over_width_only", "static void view_ig(",
     "int64_t ne = (int64_t)cam->width * cam->height;", "int64_t ne = (int64_t)cam->width;"),
    ("corner_grid_spacing_over_w", "void orc_camera_consts(",
     "cc->xstep = w > 1 ? (float)(2.0 * dh / (double)(w - 1)) : 0.0f;",
     "cc->xstep = w > 1 ? (float)(2.0 * dh / (double)w) : 0.0f;"),
    ("full_angle_tangent", "void orc_camera_consts(",
     "double dh = (double)cam->max_range * tan((double)cam->fov_h * 0.5);",
     "double dh = (double)cam->max_range * tan((double)cam->fov_h);"),
    ("rotation_sign_error", "static void quat_to_rot_f32(", "r[2] = 2.0f * (xz + wy);", "r[2] = 2.0f * (xz - wy);"),
    ("spherical_range_not_normalised", "void orc_view_ray_f32(", "float sc = cc->zc / len;", "float sc = 1.0f;"),
    ("origin_not_subtracted", "void orc_view_ray_f32(",
     "o[a] = (pose[a] - m->origin[a]) * inv_s;", "o[a] = pose[a] * inv_s;"),
    ("rays_ordered_column_major", "void orc_view_rays(",
     "int64_t k = (int64_t)j * cam->width + i;", "int64_t k = (int64_t)i * cam->height + j;"),
    ("trajectory_drops_last_pose", "int orc_traj_ig(",
     "for (int32_t k = offsets[t]; k < offsets[t + 1]; ++k) {",
     "for (int32_t k = offsets[t]; k < offsets[t + 1] - 1; ++k) {"),
    ("centre_grid_without_half_step", "void orc_camera_consts(",
     "cc->x0 = (float)(-dh + dh / (double)w);", "cc->x0 = (float)(-dh);"),
    ("spherical_length_without_z", "void orc_view_ray_f32(",
     "float len = sqrtf((cx * cx + cy * cy) + cz * cz);", "float len = sqrtf(cx * cx + cy * cy);"),
    ("steps_exclude_the_occluding_voxel", "static int visit_gain(",
     "acc->steps += 1;", "acc->steps += occ ? 0 : 1;"),
    ("tie_gap_always_zero", "double orc_min_tie_gap(", "  free(c);\n  return best;", "  free(c);\n  return 0.0;"),
    ("tie_gap_never_reports_ties", "double orc_min_tie_gap(", "  free(c);\n  return best;",
     "  free(c);\n  return INFINITY;"),
    ("ray_sum_in_fp32", "/* Gain g(v) of one voxel", "  double ig;", "  float ig;"),
    ("view_sum_in_fp32", "static void view_ig(", "double sum = 0.0;", "float sum = 0.0f;"),
    ("thread_ranges_skip_a_view", "int orc_views_ig(",
     "n_views * t / n_threads, n_views * (t + 1) / n_threads,",
     "n_views * t / n_threads + (t > 0), n_views * (t + 1) / n_threads,"),
]


def plant(src: str, anchor: str, text: str, planted: str) -> str:
    i = src.index(text, src.index(anchor))
    return src[:i] + planted + src[i + len(text):]


def first_failing_pin(lib_path: str):
    """Name of the first pin that fails against the build at lib_path, or None."""
    with oracle.using_library(lib_path):
        for name, kw in PINS:
            try:
                getattr(pins, name)(oracle, **kw)
            except Exception:
                return f"{name}{kw or ''}"
    return None


def build_copy(tmp_path, source: str) -> str:
    c = tmp_path / "oracle_copy.c"
    c.write_text(source)
    return compile_source(str(c), str(tmp_path / "liboracle_copy.so"))


def test_unmodified_copy_passes_every_pin(tmp_path):
    assert first_failing_pin(build_copy(tmp_path, open(SRC).read())) is None


@pytest.mark.parametrize("name,anchor,text,planted", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_a_pin_catches_the_planted_mistake(tmp_path, name, anchor, text, planted):
    src = open(SRC).read()
    assert src.count(anchor) == 1
    mutated = plant(src, anchor, text, planted)
    assert mutated != src
    assert first_failing_pin(build_copy(tmp_path, mutated)) is not None, f"no pin catches {name}"
