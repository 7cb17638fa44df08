"""Host logic of bench.py that the measurement depends on, without a GPU:
the clock record's throttle detection, the source hash that keeps the DRAM
traffic figure tied to the kernels it was captured for, the HBM peak lookup,
and the algorithmic flop counts behind the roofline."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _summary_of(tmp_path, lines):
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(lines) + "\n")
    c = bench.ClockSampler(0)
    c.proc, c.path = _Proc(), str(path)
    return c.summary()


def test_clock_summary_median_max_and_reasons(tmp_path):
    ok = "0, {sm}, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, {cap}"
    lines = [ok.format(sm=sm, cap="Not Active") for sm in (2070, 2055, 1995)]
    lines.append(ok.format(sm=1980, cap="Active"))
    lines.append("garbage line")
    s = _summary_of(tmp_path, lines)
    assert s["sm_mhz"] == pytest.approx((2055 + 1995) / 2) and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 4


def test_clock_summary_reports_thermal_and_hw_slowdown(tmp_path):
    line = "0, 1500, 2070, 1300.0, 0x48, Active, Not Active, Active, Not Active"
    s = _summary_of(tmp_path, [line, line])
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples_is_none(tmp_path):
    assert _summary_of(tmp_path, ["not, a, number"]) is None


def test_traffic_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("// a kernel\n__global__ void f(int *x) { x[0] = 1; } /* done */\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "TRAFFIC_SOURCES", ["k.cu"])
    h0 = bench.sources_sha256()
    src.write_text("// the same kernel, reworded comment\n__global__ void f(int *x)\n{ x[0] = 1; }\n")
    assert bench.sources_sha256() == h0
    src.write_text("__global__ void f(int *x) { x[0] = 2; }\n")
    assert bench.sources_sha256() != h0


def test_hbm_peak_from_measured_file_or_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_hbm_gbs()[0] == 6800.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6783.1}))
    v, src = bench.measured_hbm_gbs()
    assert v == 6783.1 and "MEASURED_PEAKS" in src


def test_flop_and_instruction_counts_are_consistent():
    # 100 algorithmic flops per update, split 48 / 52 between the kernels.
    # With every Pi-row product an FP64 FMA an update takes 56 FP64
    # instructions: the 20 that stay on the FP64 pipe plus one per
    # fixed-point product, less the corrector's two unit-coefficient terms
    # (Pi itself, real and imaginary part), which an FMA chain takes as its
    # starting value
    assert bench.FLOPS_PREDICTOR_POINT + bench.FLOPS_CORRECTOR_POINT == bench.FLOPS_PER_UPDATE == 100
    assert bench.BYTES_PER_UPDATE_ALG == 64
    assert bench.FP64_INSTR_PER_UPDATE + bench.FIXED_POINT_PRODUCTS_PER_UPDATE - 2 == 56


def test_issue_roofline_constants():
    # the ncu capture's warp instructions per launch of the 8192 x 128
    # workload at step 40192: 851 thread instructions per mid-point and 1430 per node
    import bench
    pred = 32 * bench.NCU_TRAFFIC["predictor_inst"] / (8191 * 128)
    corr = 32 * bench.NCU_TRAFFIC["corrector_inst"] / (8190 * 128)
    assert round(pred) == 851 and round(corr) == 1430
    assert bench.NUM_SMS * bench.ISSUE_PER_CLK_SM * 2.07e9 == pytest.approx(1.2586e12, rel=1e-4)


def test_run_gpu_does_not_rebind_the_clock_sampler():
    # run_gpu samples clocks with the object it binds to `clk` before the
    # timed region; no later assignment may rebind that name
    import ast
    import inspect
    import bench
    tree = ast.parse(inspect.getsource(bench.run_gpu))
    targets = [t.id for node in ast.walk(tree) if isinstance(node, (ast.Assign, ast.AugAssign))
               for t in (node.targets if isinstance(node, ast.Assign) else [node.target]) if isinstance(t, ast.Name)]
    withs = [it.optional_vars.id for node in ast.walk(tree) if isinstance(node, ast.With) for it in node.items
             if isinstance(it.optional_vars, ast.Name)]
    assert targets.count("clk") + withs.count("clk") == 1, (targets.count("clk"), withs.count("clk"))


def test_batch_form_letters_name_the_binding_forms():
    # each --batch-mode letter must label its results with the form it runs
    from paper_1206_0270_gb300 import teuk as T
    names = {k: T.BATCH_FORMS[i] for k, i in bench.BATCH_FORM_INDEX.items()}
    assert names["1"].startswith("per-job")
    assert names["0"] == "multi-job launches, one CTA per tile"
    assert names["p"].startswith("persistent")
    assert len(T.BATCH_FORMS) == 4


def test_optional_block_keeps_the_line_when_a_part_fails():
    assert bench.optional_block(lambda: dict(value=1.0)) == dict(value=1.0)

    def broken():
        raise RuntimeError("CUDA error: out of memory")
    out = bench.optional_block(broken)
    assert out == {"error": "RuntimeError: CUDA error: out of memory"}
    import json
    json.dumps({"value": 1.0, "serving": out})                 # still one printable JSON line


def test_reference_arm_prints_the_contract_line(capsys, monkeypatch):
    # `bench.py --impl reference` times the oracle on the host cores and prints
    # one JSON line with the headline metric, impl, cpu_baseline and a
    # copy-free e2e block (here 2 timed steps of 2 oracle time steps each)
    import argparse
    import json
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    args = argparse.Namespace(steps=2, warmup=1, ref_steps=2)
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["steps"] == 2 and line["warmup"] == 1 and line["n_gpus"] == 1
    assert line["higher_is_better"] is True and line["value"] > 0
    assert line["config"]["workload"] == bench.WORKLOAD
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == dict(value=line["value"], unit=bench.UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0)


def test_reference_arm_other_ranks_exit_quietly(capsys, monkeypatch):
    import argparse
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(argparse.Namespace(steps=2, warmup=1, ref_steps=2)) == 0
    assert capsys.readouterr().out == ""
