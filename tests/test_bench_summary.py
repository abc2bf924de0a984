"""Host logic of bench.py's compact summary block (the last key of the JSON line).

The block restates the line's key figures in a few kilobytes, so that the part of
a long line that a tail of the output keeps still carries the headline rooflines,
the FP32 arm and ratios, the error against the FP64 oracle and the compute-bound
variants. Built here from a synthetic line of the same structure; no GPU.
"""
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _line():
    ratio = {"contract_speedup_split_bf16_vs_fp32": 7.5123456, "step_speedup_split_bf16_vs_fp32": 2.5123456,
             "step_speedup_bound": 2.4123456, "kernel_ms": {"x": 1.0}}
    return {
        "metric": "field voxels/s", "value": 8.512345678e10, "ms_per_step": 0.19712345,
        "step_roofline": {"bytes": 1000098816, "ms": 0.147, "frac": 0.7456789},
        "roofline": {"kernel": "contract_tc_kernel", "frac": 0.8612345, "achieved": 5855.6,
                     "traffic": 616792064, "algorithmic_bytes": 600155136},
        "timeline_us": {"phases": [0.0, 5.2], "contraction": [4.9, 101.5]},
        "fp32": {"value": 5.53e10, "ms_per_step": 0.3033, "kernel_ms": {"contract_ms": 0.212}},
        "split_bf16_vs_fp32": {"step": 1.54, "contraction": 2.07, "note": "long text " * 20},
        "error_vs_fp64": {"voxels": 16777216,
                          "split_bf16": {"rel_l2": [6.7e-06, 9.3e-05, 7.4e-06], "max_abs_over_max": [3e-6, 6e-5, 3e-6]},
                          "fp32": {"rel_l2": [4e-07, 2e-06, 4e-07], "max_abs_over_max": [1e-7, 2e-6, 1e-7]}},
        "config3": {"tiny": {"fp32": {}}, "layers_4_planes_64": ratio, "illuminations_16_128x128": ratio},
        "e2e": {"value": 4.6e9}, "cpu_baseline": {"value": 9.1e6},
        "sweep": {"value": 2.7e10, "roofline_frac": 0.85},
        "illumination": {"split_bf16": {"ms_per_step": 1.57, "contract_tflops": 420.0}},
        "points": {"window_256x256_of_4um": {"split_bf16": {"point_product_tflops": 511.0},
                                             "point_product_speedup_split_bf16_vs_fp32": 19.1}},
        "tiling": None,
        "solve": {"gpu_s": 9.97, "cpu_baseline": {"value": 120.4}},
        "surrogate": {"train_ms_per_step": 1.21, "infer_ms_per_batch": 0.494,
                      "kernel_ms_per_train_step": {"dft": 0.267, "layer": 0.445},
                      "layer_rooflines": {"hbm": {"frac": 0.48}, "tensor": {"frac": 0.38}},
                      "gpu_launches": {"train_step": 41, "infer": 15}},
    }


def test_summary_carries_the_key_figures_in_a_short_block():
    b = _bench()
    sm = b.summary(_line())
    text = json.dumps(sm)
    assert len(text) < 2500
    assert sm["ms_per_step"] == 0.1971 and sm["step_roofline_frac"] == 0.7457
    assert abs(sm["contraction"]["traffic_over_algorithmic"] - 616792064 / 600155136) < 1e-3
    assert sm["fp32"]["contract_ms"] == 0.212
    assert "note" not in sm["split_bf16_vs_fp32"]
    assert sm["error_vs_fp64"]["split_bf16_rel_l2"] == [6.7e-06, 9.3e-05, 7.4e-06]
    assert set(sm["config3"]) == {"layers_4_planes_64", "illuminations_16_128x128"}  # entries with ratios only
    assert sm["config3"]["layers_4_planes_64"]["step_speedup_split_bf16_vs_fp32"] == 2.512
    assert sm["tiling"] == {"periodic_frac": None, "mosaic_frac": None}  # a block that did not run
    assert sm["surrogate"]["layer_hbm_frac"] == 0.48


def test_significant_digit_rounding_is_recursive():
    b = _bench()
    assert b._r({"a": [1.23456789, {"b": 0.000123456}], "c": 7, "d": "x"}) == \
        {"a": [1.235, {"b": 0.0001235}], "c": 7, "d": "x"}
    assert b._get({"a": {"b": 1}}, "a", "b") == 1 and b._get({"a": 1}, "a", "b") is None
