"""Host logic of bench.py that the GPU runs rely on (no GPU): the stored kernel
choice survives a write and read, the DRAM traffic table answers only while
the kernel sources it was measured on are unchanged, the CPU-oracle sample
spreads over the energy grid, and the argument defaults match the documented
certificate thresholds."""
import importlib.util
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_choice_round_trip(tmp_path):
    b = _bench()
    choice = np.array([-1, 2, 3, -1, 0, 1, 4, 2], dtype=np.int8)
    path = tmp_path / "choice.txt"
    b.save_choice(str(path), choice, 16, 2)
    leaf, delay, back = b.load_choice(str(path))
    assert (leaf, delay) == (16, 2) and back.dtype == np.int8 and np.array_equal(back, choice)


def test_traffic_table_follows_the_kernel_sources(monkeypatch):
    b = _bench()
    kinds = list(b.TRAFFIC)
    assert "complex-fp32x2:gemm_tc" in kinds
    digest = b.kernel_digest()
    stamped = {k: (v, d) for k, (v, d) in b.TRAFFIC.items()}
    monkeypatch.setattr(b, "TRAFFIC", {k: (v, digest) for k, (v, _) in stamped.items()})
    assert all(b.traffic_per_launch(k) == stamped[k][0] for k in kinds)
    monkeypatch.setattr(b, "TRAFFIC", {k: (v, "0" * 16) for k, (v, _) in stamped.items()})
    assert all(b.traffic_per_launch(k) is None for k in kinds)
    assert b.traffic_per_launch("no-such-kernel") is None


def test_oracle_sample_spreads_over_the_grid():
    b = _bench()
    pick = np.asarray(b.oracle_pick(256, 6))
    assert len(pick) == 6 and pick.min() == 0 and pick.max() == 255 and np.all(np.diff(pick) > 0)


def test_argument_defaults(monkeypatch):
    b = _bench()
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = b.parse()
    from paper_1305_1070_gb300 import solver
    assert (a.gpus, a.steps, a.impl, a.workload) == (1, 3, "ours", b.WORKLOAD)
    assert a.warmup >= 3
    assert a.resid_max == solver.RESID_MAX and a.growth_max == solver.GROWTH_MAX


def test_stored_choice_of_the_profiles():
    """The committed tuner choice that the profile commands load: the
    benchmark's leaf size and delay, one entry per step, each a kernel the
    choice API accepts (-1 default rule, 0 large tile, 1 small tile, 2 tensor
    cores, 3 one CTA per block, 4 extra-large tile), tensor cores present."""
    b = _bench()
    path = os.path.join(ROOT, "paper_1305_1070_gb300", "choices", "superlattice_512x128_fp32x2_leaf16_delay2.txt")
    leaf, delay, choice = b.load_choice(path)
    saved = sys.argv
    try:
        sys.argv = ["bench.py"]
        a = b.parse()
    finally:
        sys.argv = saved
    assert (leaf, delay) == (a.leaf, a.delay) == (16, 2)
    assert choice.size == 356 and choice.min() >= -1 and choice.max() <= 4
    assert (choice == 2).sum() > 0 and (choice == 3).sum() > 0


def test_profile_commands_use_existing_options():
    """Every `python bench.py ...` command recorded under profiles/ names only
    options that bench.py accepts, so the summaries stay reproducible from
    the committed files."""
    import glob
    import re
    b = _bench()
    saved = sys.argv
    try:
        sys.argv = ["bench.py"]
        known = set(vars(b.parse()).keys())
    finally:
        sys.argv = saved
    seen = 0
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        for line in open(path):
            if "python bench.py" not in line:
                continue
            for opt in re.findall(r"\s--([a-z][a-z0-9-]*)", line.split("python bench.py", 1)[1]):
                assert opt.replace("-", "_") in known, (os.path.basename(path), opt)
                seen += 1
    assert seen > 10


def test_traffic_table_matches_its_profile_summary():
    """bench.py's DRAM traffic per launch is the figure of the committed
    summary (profiles/traffic_...md, GB per 128-energy launch), kind by kind,
    and every entry carries one digest."""
    import re
    b = _bench()
    path = os.path.join(ROOT, "profiles", "traffic_fp32x2_superlattice_512x128_4_energies.md")
    rows = {}
    for line in open(path):
        m = re.match(r"\|\s*(gemm_tc|gemm_direct|gemm|gemm_small|inverse|delay)\b[^|]*\|[^|]*\|\s*(\d+)\s*\|"
                     r"\s*([\d.]+)\s*\|\s*([\d.]+)\s*\|", line)
        if m:
            rows[m.group(1)] = float(m.group(4))
    assert set(rows) == {"gemm_tc", "gemm_direct", "gemm", "gemm_small", "inverse", "delay"}
    for kind, gb in rows.items():
        value, _ = b.TRAFFIC["complex-fp32x2:" + kind]
        assert abs(value / 1e9 - gb) <= 0.0005 + 1e-9, (kind, value, gb)
    assert len({d for _, d in b.TRAFFIC.values()}) == 1
