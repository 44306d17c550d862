"""bench.py's JSON line is assembled by a pure function; check it on the
CPU with made-up timings so that a formatting slip cannot lose a GPU run."""

import argparse
import json

import bench


def _args(**kw):
    a = argparse.Namespace(gpus=1, steps=20, warmup=3, impl="gff", increments=4, cpu_applies=3, grid=128)
    for k, v in kw.items():
        setattr(a, k, v)
    return a


def _raw():
    return {"ms64": 20 * 3.0, "ms32": 20 * 0.4, "msd": 20 * 3.1, "k64": [1.5, 0.8, 0.7], "k32": [0.15, 0.12, 0.1],
            "e2e_s": 20 * 0.01, "xbytes": 9 * 128 ** 3 * 8,
            "clocks": {"sm_mhz": 1965.0, "sm_max_mhz": 2070.0, "reasons": []},
            "increment": {"workload": "w", "fp64": {"s_per_increment": 0.5}, "mixed": {"s_per_increment": 0.2}},
            "cpu": {"value": 0.2, "unit": "applies/s", "cores": 1, "kind": "oracle", "sample": "s"}}


def test_line_has_the_contract_keys():
    line = bench.build_line(_args(), 1, _raw(), {"hbm_gbs": 7000.0}, "measured")
    s = json.dumps(line)
    assert json.loads(s)["metric"] == bench.METRIC
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
              "gpu_launches", "clocks"):
        assert k in line, k
    assert abs(line["value"] - 1000.0 / 3.0) < 1e-9
    assert line["config"]["workload"]
    r = line["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in r
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert line["gpu_launches"] == 60
    assert line["e2e"]["h2d_bytes_per_step"] == 9 * 128 ** 3 * 8


def test_roofline_bytes_and_bound():
    b64 = bench.kernel_bytes_per_voxel(128, 8)
    assert abs(sum(b64) - (648 + 72 + 72 + 4 * 9 * 16 * 65 / 128)) < 1e-9
    b32 = bench.kernel_bytes_per_voxel(128, 4)
    assert abs(sum(b32) * 2 - sum(b64)) < 1e-9
    # slow FP64 kernels are ALU-bound against 1.25 TF/s, the FP32 variant HBM-bound
    line = bench.build_line(_args(), 1, _raw(), {"hbm_gbs": 7000.0}, "measured")
    assert line["roofline"]["bound"] == "alu"
    assert line["variants"]["fp32_apply"]["roofline"]["bound"] == "hbm"


def test_workload_config_names_the_sizes():
    c = bench.workload_config(64)
    assert c["grid"] == [64, 64, 64] and "64^3" in c["workload"]


def test_algorithmic_bytes_and_flops_per_voxel_at_128():
    """The per-voxel figures the roofline divides by: bytes of each apply
    kernel (every field read or written once) and the 5 n log2 n FLOP
    convention, with the z pass transforming two fields per tensor row."""
    b64, b32 = bench.kernel_bytes_per_voxel(128, 8), bench.kernel_bytes_per_voxel(128, 4)
    assert abs(b64[0] - 793.125) < 1e-9 and abs(b64[1] - 146.25) < 1e-9 and abs(b64[2] - 145.125) < 1e-9
    assert abs(sum(b64) - 1084.5) < 1e-9 and abs(sum(b32) - 542.25) < 1e-9
    fl = bench.kernel_flops_per_voxel(128)
    fr = 65 / 128
    assert abs(fl[0] - (162 + 9 * (2.5 * 7 + 5 * 7 * fr))) < 1e-9
    assert abs(fl[1] - (6 * 2 * 5 * 7 * fr + 72 * fr)) < 1e-9
    assert abs(fl[2] - 9 * (2.5 * 7 + 5 * 7 * fr)) < 1e-9
