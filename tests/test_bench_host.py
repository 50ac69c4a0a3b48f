"""Host-side logic of bench.py: the algorithmic work counts behind the roofline
fractions, and the parsing of the clock samples taken during the timed region."""
import os
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_flop_counts():
    # per complex multiply-add 8 flop; projected layer at (M, K) = (64, 8), T = 10:
    # 10 layers of two K^2 M contractions, then the setup K^2 M / 2 + K^3 / 6 + K^2 M
    K, M, T = 8, 64, 10
    assert bench.flops_per_instance(K, M, T, 1) == pytest.approx(
        8 * (T * 2 * K * K * M + K * K * M / 2 + K ** 3 / 6 + K * K * M))
    assert bench.flops_per_instance(K, M, T, 1) == pytest.approx(705194.667, rel=1e-9)
    assert bench.flops_per_instance(K, M, T, 0) == 8 * T * 2 * K * K * M  # paper layer: no setup
    # train step: the forward, the loss residual and its gradient, T reverse layers
    assert bench.train_flops_per_instance(K, M, T) == pytest.approx(1426090.667, rel=1e-9)


def test_mma_counts():
    # split FP16: 24 m16n8k16 per 8 x 64 contraction; two per layer, the final residual,
    # the Gram matrix (one residual) and Q / Q^T (48)
    assert bench.mma_per_instance_f16(10) == (48 * 10 + 96, 0)
    assert bench.mma_per_instance_f16(0) == (96, 0)
    # split TF32: 48 m16n8k8 per contraction
    assert bench.mma_per_instance(10) == 96 * 10 + 192


def test_tcgen05_counts():
    # transposed tcgen05 kernel at 32 x 256: the Gram matrix and Q^T in the setup, 16
    # M = N = 128 K = 16 products each; a layer: the residual (16 of them) and the
    # update (8 at N = 128 for Q hi, 8 at N = 64 for Q lo x E hi); the final residual
    # (16) only when the residual is asked for.  2 M N K flop per product.
    big, small = 2 * 128 * 128 * 16, 2 * 128 * 64 * 16
    f, slots = bench.tcgen05_flop_per_instance(10, False)
    assert slots == 2 * 16 + 10 * (16 + 8 + 8) == 352
    assert f == (2 * 16 + 10 * (16 + 8)) * big + 10 * 8 * small == 163_577_856
    f_r, slots_r = bench.tcgen05_flop_per_instance(10, True)
    assert slots_r - slots == 16 and f_r - f == 16 * big
    f1, slots1 = bench.tcgen05_flop_per_instance(1, False)
    assert slots1 == 64 and f1 == 56 * big + 8 * small


def test_fp32_peak():
    assert bench.fp32_peak_tflops() == pytest.approx(152 * 128 * 2 * 2.070e9 / 1e12)
    bench.set_fp32_peak(148, 1965.0, "test")
    assert bench.fp32_peak_tflops() == pytest.approx(148 * 128 * 2 * 1.965e9 / 1e12)
    bench.set_fp32_peak(152, 2070.0, "default")


def _summary(lines):
    fd, path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("\n".join(lines) + "\n")
    cs = bench.ClockSampler(0)
    cs.proc, cs.path = object(), path  # as if nvidia-smi had written the samples
    return cs.summary()


def test_clock_summary_under_load_and_reasons():
    idle = "0, 1200, 2070, 150.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    busy = "0, {}, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, {}"
    s = _summary([idle, busy.format(2070, "Not Active"), busy.format(2055, "Active"),
                  busy.format(2070, "Not Active"), idle])
    assert s["samples"] == 5 and s["samples_under_load"] == 3
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    hot = "0, 1500, 2070, 1000.0, 0x0, Not Active, Active, Not Active, Not Active"
    assert _summary([hot])["reasons"] == ["hw_thermal_slowdown"]


def test_clock_summary_without_samples():
    assert _summary(["garbage"]) is None
    cs = bench.ClockSampler(0)
    assert cs.summary() is None  # nvidia-smi never started


def test_cpu_baseline_on_a_small_sample():
    """The oracle leg of the bench: one-thread rate first, then all cores over
    contiguous ranges; the objectives it hands back are the oracle's own."""
    import numpy as np
    import oracle
    from paper_2304_12745_gb300 import channels as ch
    H = ch.lognormal(96, 8, 64, seed=2)
    t = ch.targets(96, 8)
    mu = ch.fixed_workload_steps(10)
    cb, (lo, obj) = bench.cpu_baseline(H, t, mu, budget_s=0.3)
    assert cb["kind"] == "oracle" and cb["unit"] == "precoders/s"
    assert cb["cores"] == (os.cpu_count() or 1)
    assert cb["value"] > 0 and cb["single_thread_value"] > 0 and cb["sample"]
    n = len(obj)
    _, ref, _, st = oracle.batch_forward(1, H[lo:lo + n].astype(np.complex128),
                                         t[lo:lo + n].astype(np.float64), mu.astype(np.float64))
    assert np.all(st == 0) and np.array_equal(obj, ref)


def test_profile_commands_parse():
    """Every `python bench.py ...` command in profiles/ (continuation lines joined,
    comments dropped) is a valid invocation of the committed bench, also with the
    flags the summaries name for reproducing older captures."""
    import glob
    import re
    cmds = []
    for f in glob.glob(os.path.join(ROOT, "profiles", "*")):
        text = open(f).read().replace("\\\n", " ")
        for line in text.splitlines():
            m = re.search(r"python bench\.py([^#\n]*)", line)
            if m:
                cmds.append((os.path.basename(f), m.group(1).split()))
    assert len(cmds) >= 10
    for name, argv in cmds:
        for extra in ([], ["--tf32"], ["--ffma"]):
            bench._parser().parse_args(argv + extra)  # SystemExit on an unknown flag
