"""Host-side bookkeeping of bench.py (no GPU): the byte models behind the
roofline, the recorded-traffic lookup that guards the ncu numbers, the peak
lookup and the whole-job rate."""
import json
import os

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_unpruned_model_is_216_fields_per_step():
    # one field F = N^2 (N/2+1) complex; 54 F per stage, 4 stages
    for N, dtype, c in ((512, 0, 8), (256, 1, 16), (1024, 0, 8)):
        F = N * N * (N // 2 + 1) * c
        assert bench.unpruned_step_bytes(N, dtype) == 216 * F
    assert bench.unpruned_step_bytes(512, 0) == 116_417_101_824


def test_pruned_pass_bytes_structure():
    N = 512
    K = (N - 1) // 3
    Kz = K + 1
    stages = [bench.pass_bytes(N, 0, s) for s in range(4)]
    # the transform passes move the same bytes at every stage; only the update differs
    for s in range(1, 4):
        assert stages[s][:5] == stages[0][:5]
    # z pass: six packed half-lines in, three out, N^2 lines of Kz modes
    assert stages[0][2] == 9 * N * N * Kz * 8
    # the middle stages read and write the accumulator as well
    assert stages[1][5] == stages[2][5] > stages[0][5] == stages[3][5]
    pruned = sum(sum(p) for p in stages)
    assert pruned < bench.unpruned_step_bytes(N, 0)
    # FP64 doubles every term; F32 with FP64 accumulators only the update's
    st64 = [bench.pass_bytes(N, 1, s) for s in range(4)]
    assert all(a == 2 * b for s in range(4) for a, b in zip(st64[s], stages[s]))
    acc = [bench.pass_bytes(N, 2, s) for s in range(4)]
    assert all(acc[s][:5] == stages[s][:5] and acc[s][5] > stages[s][5] for s in range(4))


def _profile_lines(N):
    with open(os.path.join(ROOT, "profiles", f"dram_fp32_{N}.txt")) as f:
        return f.read().splitlines()


@pytest.mark.parametrize("N,lo", [(256, 0.7), (512, 0.97), (1024, 0.97)])
def test_recorded_dram_traffic_agrees_with_the_byte_model(N, lo):
    # the ncu DRAM bytes per launch kept in profiles/ are at most 3 % above
    # the algorithmic bytes of each pass (averaged over the four stages): no
    # pass re-reads what it has read once.  At 512^3 (a working set many
    # times the 129 MB L2; 1024^3 likewise) they are also at most 3 % below; at 256^3 part of
    # each pass's input is still in L2 from the pass before, so less reaches
    # DRAM
    lines = _profile_lines(N)
    avg = [sum(bench.pass_bytes(N, 0, s)[i] for s in range(4)) / 4 for i in range(6)]
    seen = 0
    for line in lines:
        f = line.split()
        if len(f) == 4 and f[0] == "traffic":
            i = bench.PASS_NAMES.index(f[1])
            assert lo < float(f[3]) / avg[i] < 1.03, (f[1], float(f[3]), avg[i])
            seen += 1
    assert seen == 6


def test_recorded_traffic_is_used_only_for_the_profiled_sources(monkeypatch):
    lines = _profile_lines(512)
    sha = [l.split()[1] for l in lines if l.startswith("source_sha256:")][0]
    rec = {}
    for line in lines:
        f = line.split()
        if len(f) == 4 and f[0] == "traffic":
            rec[f[1]] = (int(f[2]), float(f[3]))
    name, (variant, value) = "p3_z_cross", rec["p3_z_cross"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: sha)
    assert bench.recorded_traffic(512, name, variant) == value
    assert bench.recorded_traffic(512, name, variant + 1) is None  # another launch variant
    assert bench.recorded_traffic(48, name, variant) is None  # no summary for this mesh
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 64)
    assert bench.recorded_traffic(512, name, variant) is None  # kernels changed since


def test_kernel_source_hash_covers_the_step_kernels(tmp_path, monkeypatch):
    h0 = bench.kernel_source_hash()
    assert len(h0) == 64 and h0 == bench.kernel_source_hash()
    csrc = tmp_path / "paper_1607_00850_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in bench.KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1607_00850_gb300", "csrc", name), "rb") as f:
            (csrc / name).write_bytes(f.read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_source_hash() == h0
    (csrc / "dns_passes.cuh").write_bytes((csrc / "dns_passes.cuh").read_bytes() + b"\n")
    assert bench.kernel_source_hash() != h0


def test_measured_peak_or_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6789.0}))
    assert bench.measured_peaks() == (6789.0, "measured")


def test_whole_job_rate_counts_every_replica():
    assert bench.whole_job_rate(1, 512, 20, 2.0) == 512.0 ** 3 * 10
    assert bench.whole_job_rate(4, 64, 10, 1.0) == 4 * 64.0 ** 3 * 10
    assert bench.max_over_ranks(3.5) == 3.5


def test_step_flops_grow_as_n3_log_n():
    r = bench.step_flops(1024) / bench.step_flops(512)
    assert 8.0 < r < 8.0 * (10 / 9) * 1.05


def test_step_launch_count_follows_the_plan():
    assert bench.step_launches([7, 7, 9, 3, 0]) == 24
    assert bench.step_launches([7, 7, 9, 3, 7]) == 24
    assert bench.step_launches([9, 9, 14, 8, 9]) == 24  # half-width column variants
    assert bench.step_launches([7, 7, 9, 3, bench.FUSED_P5_FROM]) == 20


def test_fused_variant_offset_matches_the_library():
    # plan[4] >= NCOLV selects a fused x-forward + update variant in the
    # library (dns_api.cu); bench.py counts launches with the same offset
    import re
    with open(os.path.join(ROOT, "paper_1607_00850_gb300", "csrc", "dns_internal.h")) as f:
        ncolv = int(re.search(r"NCOLV\s*=\s*(\d+)", f.read()).group(1))
    assert bench.FUSED_P5_FROM == ncolv
