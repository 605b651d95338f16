"""CPU checks of host-side logic: the seeded DIA input generator, the
traffic lookup of bench.py against the committed ncu summary, and the
bench's argument parsing for the sweep modes."""
import hashlib
import os
import sys

import numpy as np

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_dia_matrix_generator():
    n = 500
    off, val = synth.dia_matrix(n, [7, -3, 0, 7, -499], seed=4, zero_rate=0.0)
    assert off.tolist() == [-499, -3, 0, 7]          # sorted, duplicates merged
    assert val.shape == (4, n)
    i = np.arange(n)
    for k, o in enumerate(off):
        inside = (i + o >= 0) & (i + o < n)
        assert np.all(np.isnan(val[k, ~inside]))       # padding outside the matrix
        assert np.all(val[k, inside] != 0.0)           # no zeros without zero_rate
        assert np.all(np.abs(val[k, inside]) <= 1.0)
    off2, val2 = synth.dia_matrix(n, [7, -3, 0, -499], seed=4, zero_rate=0.0)
    assert np.array_equal(val, val2, equal_nan=True)   # seeded
    _, vz = synth.dia_matrix(n, [0], seed=4, zero_rate=0.5)
    frac = np.mean(vz == 0.0)
    assert 0.4 < frac < 0.6
    assert synth.paper_stencil_offsets(1000, 3) == [-100, -10, -1, 0, 1, 10, 100]
    assert synth.paper_stencil_offsets(10000, 2) == [-100, -1, 0, 1, 100]


def test_profiled_traffic_matches_source_hash(tmp_path, monkeypatch):
    import bench
    root = tmp_path
    (root / "profiles").mkdir()
    (root / "paper_2105_04937_gb300" / "csrc").mkdir(parents=True)
    h = hashlib.sha1()
    for name in bench.KERNEL_SOURCES:
        src = f"// {name}\n".encode()
        (root / "paper_2105_04937_gb300" / "csrc" / name).write_bytes(src)
        h.update(src)
    sha = h.hexdigest()[:16]
    (root / "profiles" / "mhdc_spmv_f64_stencil27_128.md").write_text(
        f"text\ntraffic: 1 350833152 {sha}\ntraffic: 5 350264832 0000000000000000\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.profiled_traffic(1) == 350833152
    assert bench.profiled_traffic(5) is None      # captured for another source
    assert bench.profiled_traffic(3) is None      # not captured
    (root / "paper_2105_04937_gb300" / "csrc" / "spmv_tma.cu").write_bytes(b"// changed\n")
    assert bench.profiled_traffic(1) is None      # a kernel source changed since


def test_bench_parses_sweep_options(monkeypatch):
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", "--sweep", "stencil", "--sizes", "1e4,2e4",
                                      "--nb-n", "5e4", "--out", "x.jsonl"])
    a = bench.parse()
    assert a.sweep == "stencil" and a.sizes == "1e4,2e4" and a.nb_n == 5e4 and a.out == "x.jsonl"
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.sweep is None and a.gpus == 1 and a.warmup >= 3 and a.impl == "ours"


def test_bench_precision_bound_equals_the_oracles():
    import bench
    import oracle
    rng = np.random.default_rng(3)
    terms = rng.integers(1, 80, 1000).astype(np.float64)
    absr = rng.uniform(0, 10, 1000)
    for dt in ("f32", "bf16"):
        assert np.allclose(bench.precision_bound(dt, terms, absr),
                           oracle.bound_vs_exact(absr, terms, dt), rtol=1e-12, atol=0)
    assert np.array_equal(bench.precision_bound("f64", terms, absr), 1e-12 * absr)
