"""The pins of the numpy oracles catch planted mistakes (CPU; no GPU).

As test_oracle_mutants.py does for the C oracle: each case plants one
plausible mistake into a copy of one numpy oracle module -- Eq. 3 and the
IG cost (``oracle/idw.py``), the map update (``oracle/insert.py``), the
endpoint-grid density (``oracle/endpoints.py``) or the surrogate
(``oracle/surrogate.py``) -- loads the copy as a module of the ``oracle``
package, puts it in place of the module its pin file tests, and runs every
pin of that file (parametrisations expanded): at least one must fail.  An
unmodified copy must pass them all.
"""

import importlib.util
import inspect
import warnings

import numpy as np
import pytest

import oracle
import test_endpoints_oracle
import test_idw_oracle
import test_insert_oracle
import test_surrogate_oracle
import test_workload
from oracle import endpoints, idw, insert, surrogate
from workload import poses, scenes, trajectories

# module -> (its pin file, the name the pin file binds it to); the perspective sampler of Eq. 1
# and the look-at orientation are inputs, not oracle arithmetic, but Eq. 1 is the paper's
TARGETS = {
    "idw": (idw, test_idw_oracle, "I"),
    "insert": (insert, test_insert_oracle, "I"),
    "endpoints": (endpoints, test_endpoints_oracle, "E"),
    "surrogate": (surrogate, test_surrogate_oracle, "S"),
    "poses": (poses, test_workload, "poses"),
    "scenes": (scenes, test_workload, "scenes"),
    "trajectories": (trajectories, test_workload, "trajectories"),
}

# (target, name, text, planted text): the first occurrence of text is replaced
MUTANTS = [
    ("idw", "distance_weight_grows_with_distance", "w = d ** (-float(p))", "w = d ** float(p)"),
    ("idw", "power_applied_to_squared_distance", "w = d ** (-float(p))", "w = d ** (-2.0 * float(p))"),
    ("idw", "coincident_points_not_averaged", "return float(np.mean(g[hit]))", "return float(g[hit][0])"),
    ("idw", "weights_not_normalised", "return float(np.sum(g * w) / np.sum(w))", "return float(np.sum(g * w))"),
    ("idw", "oldest_id_weighs_most", "total += idw(query, persp, g, p) / (n_b - u)",
     "total += idw(query, persp, g, p) / (u + 1)"),
    ("idw", "partial_buffer_not_aligned_to_newest", "u = n_b - n + m", "u = m"),
    ("idw", "fov_from_full_angle", "np.float32(math.tan(float(np.float32(fov_h)) * 0.5))",
     "np.float32(math.tan(float(np.float32(fov_h))))"),
    ("idw", "poi_direction_rotated_by_r_not_its_transpose",
     "c = [f32(f32(f32(R[0][k] * v[0]) + f32(R[1][k] * v[1])) + f32(R[2][k] * v[2])) for k in range(3)]",
     "c = [f32(f32(f32(R[k][0] * v[0]) + f32(R[k][1] * v[1])) + f32(R[k][2] * v[2])) for k in range(3)]"),
    ("idw", "optical_axis_sign_error", "2 * (x * z + w * y)", "2 * (x * z - w * y)"),
    ("idw", "cost_adds_o_and_g", "term = w_i / (O * G + eps)", "term = w_i / (O + G + eps)"),
    ("idw", "cost_drops_last_state", "term[offsets[t]:offsets[t + 1]].sum()",
     "term[offsets[t]:offsets[t + 1] - 1].sum()"),
    ("insert", "miss_likelihood_not_complemented", "b = (f32(1.0) - P) * (f32(1.0) - p)",
     "b = (f32(1.0) - P) * p"),
    ("insert", "no_clamping", "return np.where(q < lo, lo, np.where(q > hi, hi, q)).astype(np.float32)",
     "return q.astype(np.float32)"),
    ("insert", "hit_voxels_also_missed", "return hits, misses - hits", "return hits, misses"),
    ("insert", "rays_aimed_at_voxel_corners", "d = (e.astype(np.float32) + f32(0.5)) - o",
     "d = e.astype(np.float32) - o"),
    ("insert", "range_compared_unsquared", "p = p[r2 <= f32(max_range) * f32(max_range)]",
     "p = p[r2 <= f32(max_range)]"),
    ("insert", "hit_update_uses_miss_likelihood", "flat[h] = update_f32(flat[h], p_hit, p_min, p_max)",
     "flat[h] = update_f32(flat[h], p_miss, p_min, p_max)"),
    ("insert", "misses_mark_unknown_on_state_maps", "flat[m] = 1", "flat[m] = 0"),
    ("insert", "sensor_origin_not_subtracted", "o = (np.asarray(sensor, np.float32) - org) * inv_s",
     "o = np.asarray(sensor, np.float32) * inv_s"),
    ("endpoints", "full_angle_tangent", "math.tan(f(fov) * 0.5)", "math.tan(f(fov))"),
    ("endpoints", "corner_count_off_by_one", "int(math.floor((2.0 * half) / step)) + 1",
     "int(math.floor((2.0 * half) / step))"),
    ("endpoints", "half_width_as_span", "(2.0 * half) / step", "half / step"),
    ("surrogate", "conv_tap_order_transposed", "tap = (dz * 3 + dy) * 3 + dx", "tap = (dx * 3 + dy) * 3 + dz"),
    ("surrogate", "relu_mask_dropped_in_backward", "da = rnd(dxin * (acts[i] > 0))", "da = rnd(dxin)"),
    ("surrogate", "backward_rounding_not_modelled", "dh = rnd(np.outer(", "dh = (np.outer("),
    ("surrogate", "input_gradient_rounding_not_modelled", "da = rnd(dxin * (acts[i] > 0))",
     "da = (dxin * (acts[i] > 0))"),
    ("surrogate", "target_scale_ignored", "t = np.asarray(targets, np.float64) * float(target_scale)",
     "t = np.asarray(targets, np.float64)"),
    ("surrogate", "mse_gradient_factor_dropped", "dy = 2.0 * (y - t) / n", "dy = (y - t) / n"),
    ("surrogate", "adam_without_bias_correction", "mh = mk / (1.0 - beta1 ** step)", "mh = mk"),
    ("surrogate", "adam_second_moment_unsquared", "(1.0 - beta2) * g * g", "(1.0 - beta2) * g"),
    ("surrogate", "crop_samples_at_slice_starts", "fr = f32(f32(k + 0.5) / f32(n))", "fr = f32(f32(k) / f32(n))"),
    ("surrogate", "free_and_occupied_classes_swapped",
     "return 2 if v > np.float32(occ_threshold) else (1 if v < np.float32(free_threshold) else 0)",
     "return 1 if v > np.float32(occ_threshold) else (2 if v < np.float32(free_threshold) else 0)"),
    ("surrogate", "crop_codes_off_by_one", "oh.argmax(axis=-1) + 1", "oh.argmax(axis=-1)"),
    ("surrogate", "bf16_truncates", "u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16", "u = (u >> 16) << 16"),
    ("surrogate", "crop_origin_not_subtracted", "o = [f32((f32(pose[a]) - f32(origin[a])) * inv_s) for a in range(3)]",
     "o = [f32(f32(pose[a]) * inv_s) for a in range(3)]"),
    ("surrogate", "pose_features_origin_not_subtracted", "feats[a] = f32(f32(f32(pose[a]) - f32(origin[a])) / ext)",
     "feats[a] = f32(f32(pose[a]) / ext)"),
    ("poses", "eq1_square_root_radius", "np.cbrt(xr)", "np.sqrt(xr)"),
    ("poses", "eq1_direction_not_normalised", "return r_s * np.cbrt(xr)[:, None] * x / norm",
     "return r_s * np.cbrt(xr)[:, None] * x"),
    ("poses", "golden_angle_wrong", "GOLDEN_ANGLE = math.pi * (3.0 - math.sqrt(5.0))",
     "GOLDEN_ANGLE = math.pi * (3.0 + math.sqrt(5.0))"),
    ("poses", "fibonacci_heights_not_centred", "z = 1.0 - (2.0 * k + 1.0) / n", "z = 1.0 - 2.0 * k / n"),
    ("poses", "image_y_axis_up", "y = np.cross(z, x)", "y = np.cross(x, z)"),
    ("poses", "optical_axis_away_from_poi", "z = poi[None, :] - pos", "z = pos - poi[None, :]"),
    ("poses", "quaternion_conjugated", "q[k] = [0.25 * s, (m[2, 1] - m[1, 2]) / s, (m[0, 2] - m[2, 0]) / s, (m[1, 0] - m[0, 1]) / s]",
     "q[k] = [0.25 * s, (m[1, 2] - m[2, 1]) / s, (m[2, 0] - m[0, 2]) / s, (m[0, 1] - m[1, 0]) / s]"),
    ("poses", "vertical_axis_without_fallback_up", "up[vertical] = np.array([1.0, 0.0, 0.0])",
     "up[vertical] = np.array([0.0, 0.0, 1.0])"),
    ("scenes", "free_and_occupied_beta_swapped", "p[free] = rng.beta(2.0, 8.0, size=int(free.sum()))",
     "p[free] = rng.beta(8.0, 2.0, size=int(free.sum()))"),
    ("scenes", "free_beta_too_narrow", "p[free] = rng.beta(2.0, 8.0, size=int(free.sum()))",
     "p[free] = rng.beta(4.0, 16.0, size=int(free.sum()))"),
    ("scenes", "unknown_probability_not_half", "p[unknown] = 0.5", "p[unknown] = 0.45"),
    ("scenes", "occupied_overrides_unknown", "    st[unknown] = UNKNOWN\n",
     "    st[unknown & ~occupied] = UNKNOWN\n"),
    ("scenes", "unknown_half_on_the_wrong_side", "unk[:, :, n // 2:] = True", "unk[:, :, :n // 2] = True"),
    ("scenes", "box_fill_by_voxel_corners", "a = max(0, math.ceil(lo - 0.5))", "a = max(0, math.floor(lo))"),
    ("trajectories", "spline_coefficient_error", "(2.0 * p0 - 5.0 * p1 + 4.0 * p2 - p3) * t * t\n",
     "(2.0 * p0 - 4.0 * p1 + 4.0 * p2 - p3) * t * t\n"),
    ("trajectories", "spline_tangent_halved", "return 0.5 * ((2.0 * p1) + (-p0 + p2) * t",
     "return 0.5 * ((2.0 * p1) + 0.5 * (-p0 + p2) * t"),
    ("trajectories", "jitter_in_degrees_as_radians", "ang = math.radians(jitter_deg) * rng.random()",
     "ang = jitter_deg * rng.random()"),
    ("trajectories", "horizon_tilt_not_skew_symmetric",
     "K[:, 1, 0], K[:, 2, 0], K[:, 2, 1] = axis[:, 2], -axis[:, 1], axis[:, 0]",
     "K[:, 1, 0], K[:, 2, 0], K[:, 2, 1] = -axis[:, 2], axis[:, 1], -axis[:, 0]"),
]


def load_copy(module, source: str, tmp_path):
    """Load source as a module of the original's package (relative imports resolve as in the original)."""
    package, name = module.__name__.rsplit(".", 1)
    path = tmp_path / f"{name}_copy.py"
    path.write_text(source)
    spec = importlib.util.spec_from_file_location(f"{package}.{path.stem}", str(path))
    mod = importlib.util.module_from_spec(spec)
    mod.__package__ = package
    spec.loader.exec_module(mod)
    return mod


def pin_calls(pin_module):
    """(name, function, kwargs) for every pin of the file, parametrisations expanded."""
    for name in sorted(dir(pin_module)):
        fn = getattr(pin_module, name)
        if not name.startswith("test_") or not callable(fn):
            continue
        combos = [{}]
        for mark in [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]:
            argnames, argvalues = mark.args[0], mark.args[1]
            names = [a.strip() for a in argnames.split(",")] if isinstance(argnames, str) else list(argnames)
            expanded = []
            for c in combos:
                for v in argvalues:
                    vals = getattr(v, "values", v if len(names) > 1 else (v,))
                    expanded.append({**c, **dict(zip(names, vals))})
            combos = expanded
        for kw in combos:
            if "orc" in inspect.signature(fn).parameters:
                kw = {**kw, "orc": oracle}
            yield name, fn, kw


def first_failing_pin(target: str, copy, monkeypatch):
    _, pin_module, attr = TARGETS[target]
    monkeypatch.setattr(pin_module, attr, copy)
    with warnings.catch_warnings(), np.errstate(all="ignore"):
        warnings.simplefilter("ignore")    # a planted mistake may divide by zero
        for name, fn, kw in pin_calls(pin_module):
            try:
                fn(**kw)
            except Exception:
                return name
    return None


@pytest.mark.parametrize("target", sorted(TARGETS))
def test_unmodified_copy_passes_every_pin(target, tmp_path, monkeypatch):
    module = TARGETS[target][0]
    copy = load_copy(module, open(module.__file__).read(), tmp_path)
    assert first_failing_pin(target, copy, monkeypatch) is None


@pytest.mark.parametrize("target,name,text,planted", MUTANTS, ids=[f"{m[0]}-{m[1]}" for m in MUTANTS])
def test_a_pin_catches_the_planted_mistake(target, name, text, planted, tmp_path, monkeypatch):
    module = TARGETS[target][0]
    src = open(module.__file__).read()
    assert text in src
    copy = load_copy(module, src.replace(text, planted, 1), tmp_path)
    assert first_failing_pin(target, copy, monkeypatch) is not None, f"no pin catches {target}: {name}"
