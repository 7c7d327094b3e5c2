"""Host-side checks of the benchmark's bookkeeping (no GPU): the committed ncu
summaries still describe the device code bench.py reports traffic for, and the
FLOP counts behind its roofline figures have the values the summaries quote."""

import importlib.util
import os

import pytest

import afqmc_inputs as ai

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("kernel,bytes_per_launch", [("contract_fp64z_kernel", 3.89e9),
                                                     ("contract_fp64r_kernel", 16.82e9)])
def test_fp64_summaries_match_the_device_code(bench, kernel, bytes_per_launch):
    src = os.path.join(ROOT, "paper_2505_18519_gb300", "csrc", bench.FP64_SOURCE.get(kernel, "contract_fp64.cu"))
    assert bench.recorded_traffic(src, *bench.FP64_TRAFFIC[kernel]) == pytest.approx(bytes_per_launch)


def test_tensor_core_summary_is_used_only_for_its_own_device_code(bench):
    """The walker-side tensor-core summary quotes 6.34 GB per contraction; bench.py
    reports it only while the kernels' device code is the one it was taken on."""
    src = os.path.join(ROOT, "paper_2505_18519_gb300", "csrc", "contract_tc.cu")
    summary, end, start = bench.TC_TRAFFIC["contract_tcy_kernel"]
    fields = dict(line[2:].split(":", 1) for line in open(os.path.join(ROOT, "profiles", summary))
                  if line.startswith("- ") and ":" in line)
    recorded = fields["source_sha256_16"].strip().strip("`")
    got = bench.recorded_traffic(src, summary, end, start)
    if recorded == bench.kernel_digest(src, end, start):
        assert got == pytest.approx(6.34e9)
    else:
        assert got is None


def test_a_changed_kernel_voids_its_traffic(bench, tmp_path):
    src = os.path.join(ROOT, "paper_2505_18519_gb300", "csrc", "rcache.cu")
    text = open(src).read().replace("acc.x = fma(r, t.x, acc.x);", "acc.x = fma(t.x, r, acc.x);", 1)
    changed = tmp_path / "rcache.cu"
    changed.write_text(text)
    assert bench.recorded_traffic(str(changed), *bench.FP64_TRAFFIC["contract_fp64r_kernel"]) is None


def test_flop_counts_of_the_medium_workload(bench):
    spec, run = ai.CONFIGS["medium_n50"]
    assert bench.contract_flops_per_pair(spec) == pytest.approx(22.99e6, rel=1e-3)      # per-pair order
    assert bench.contract_flops_walker_side(spec, run.n_paths) == pytest.approx(16.02e6, rel=1e-3)
    assert bench.contract_flops_cached(spec) == pytest.approx(10.44e6, rel=1e-3)
    assert bench.contract_flops_refresh(spec) == pytest.approx(12.55e6, rel=1e-3)
    # the cached form's share per refreshed pair: (G + 1) matrices of 2 n_up N^2
    assert bench.contract_flops_refresh(spec) == (spec.n_chol + 1) * 2 * spec.n_up * spec.N ** 2


def test_headline_contraction_summary_gives_its_traffic(bench):
    """The headline's contraction summary records DRAM bytes per pair for the
    walker-side tensor-core kernel; bench.py reports them (scaled by pairs)
    only while the kernel's device code has the recorded digest."""
    src = os.path.join(ROOT, "paper_2505_18519_gb300", "csrc", "contract_tcw.cu")
    summary, end, start = bench.TCW_TRAFFIC
    fields = dict(line[2:].split(":", 1) for line in open(os.path.join(ROOT, "profiles", summary))
                  if line.startswith("- ") and ":" in line)
    recorded = fields["source_sha256_16"].strip().strip("`")
    got = bench.tcw_traffic(1024, 64)
    if recorded == bench.kernel_digest(src, end, start):
        assert got == pytest.approx(1837315 * 1024 * 64)
    else:
        assert got is None
