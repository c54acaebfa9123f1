"""Host-side pieces of the benchmark (no GPU): the multi-rank time reduction
on two gloo ranks, and the reference arm's JSON line (the CPU oracle)."""
import json
import os
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, ws, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    sys.path.insert(0, ROOT)
    import bench
    ms = bench.reduce_max_ms(10.0 + 5.0 * rank, ws, torch.device("cpu"))
    out[rank] = (ms, bench.job_value(1000.0, ws, ms / 4))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = 29500 + os.getpid() % 1000
        mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    # 1000 units per rank, 2 ranks, 15/4 ms per step
    assert res[0][1] == pytest.approx(2000.0 / (15.0 / 4 * 1e-3))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "DOF/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["config"]["cycles"] == 9


def test_summary_is_compact_and_last():
    """The per-form summary the benchmark appends as the line's last key
    stays small enough to survive in the last 2 KB of the output."""
    sys.path.insert(0, ROOT)
    import bench
    line = {"ms_per_step": 11.5, "value": 1.44e9, "config": bench.config_of(9, 1),
            "e2e": {"ms_per_step": 13.5, "value": 1.23e9},
            "roofline": {"kernel": "rb_half (level 0)", "frac": 0.9, "hbm_frac": 0.31,
                         "bound": "alu"},
            "cufft_dst_257": {"ms_per_step": 14.9, "relres": 1e-15, "gmg_speedup_vs_fft": 1.3},
            "mixed_precision_513": {"forms": {
                n: {"ms_per_step": 38.5, "value": 3.4e9, "outer_steps": 4,
                    "inner_cycles_per_step": 3, "relres": 8e-11, "speedup_vs_fp64_plain": 2.4}
                for n in ("fp64_plain", "fp32_ir", "bf16_ir")}},
            "batched_512": {"ms_per_step": 192.0, "value": 1.25e9, "max_relres": 9e-11,
                            "speedup_vs_one_by_one": 4.4, "speedup_vs_one_by_one_fp64": 7.8,
                            "autotuned": {"inner_cycles": 3, "chunk": 4096, "ctas": 1216}},
            "learned_257": {"runs": {"learned_v11": {"ms_per_step": 27.6, "cycles": 11},
                                     "rbgs_v22": {"ms_per_step": 12.7}},
                            "contraction": {"learned_v11": 0.136, "rbgs_v11": 0.221},
                            "levels_kept": [0, 1, 2], "speedup_learned_vs_rbgs_v22": 0.46},
            "fmg_257": {"fmg_v22": {"ms_per_step": 11.2, "cycles": 8, "speedup_vs_plain_v22": 1.03},
                        "fmg_v33": {"ms_per_step": 13.2, "cycles": 7, "speedup_vs_plain_v22": 0.87}},
            "cpu_baseline": {"value": 2.3e7, "cores": 16}}
    s = bench.summarise(line)
    assert len(json.dumps({"summary": s})) < 1800
    assert set(s) >= {"plain_fp64_257", "e2e_257", "roofline", "cufft_257", "fp32_ir_513",
                      "bf16_ir_513", "fp64_plain_513", "batch_512", "learned_257",
                      "fmg_v22_257", "oracle_cpu_257"}
